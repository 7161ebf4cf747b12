// k_aev.cu -- ANI atomic environment vectors (radial + angular symmetry
// functions with cosine cutoffs) and their position derivatives.
//
//   radial:  G_i[s_j*16 + m] += 1/4 exp(-eta_r (r_ij - R_m)^2) fc(r_ij; rc_r)
//   angular: G_i[16S + p(s_j,s_k)*32 + a*8 + z] +=
//              2 ((1 + cos(theta' - theta_z)) / 2)^zeta
//              * exp(-eta_a ((r_ij + r_ik)/2 - R_a)^2) fc(r_ij; rc_a) fc(r_ik; rc_a)
//            with cos(theta' - theta_z) = u cos(theta_z) + sqrt(1 - u^2) sin(theta_z),
//            u = 0.95 cos(theta_ijk), so no arccos is evaluated.
//   fc(r; rc) = (cos(pi r / rc) + 1)/2 = cos^2(y), y = pi r / (2 rc).
//
// Forces follow Eq. 2 of the paper, F = -dE/dr, by the chain rule from dE/dG_i
// (the network backward) through these terms.
//
// Mapping: half a warp (16 lanes) per row, the two halves of a warp in lock
// step so that shuffles stay convergent.  Radial: lanes over the neighbours of
// one species, 16 accumulators per lane, half-warp reduce-scatter (lane l ends
// with feature l).  Angular: the neighbours inside rc_a (the first entries of
// each species segment of the row's list) are staged in shared memory as unit
// vector, distance and cutoff; lanes run over the neighbour pairs of one
// species-pair block (a flat index mapped to a pair without search) with 32
// accumulators (4 shifts x 8 sectors), then reduce-scatter so that lane l owns
// features 2l and 2l+1.  Species loops are not unrolled, which keeps the code
// inside the instruction cache.  FP32 throughout; forces are summed per
// neighbour slot in shared memory and added once per slot in FP64.
#include "nnp_internal.cuh"

namespace nnp {

namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kPi = 3.14159265358979f;
constexpr int kBwdWarps = 4;  // rows (warps) per k_aev_bwd block

// fc = cos^2(y), dfc/dr = -2 k sin(y) cos(y), y = k r, k = pi / (2 rc), from
// the Taylor series of cos and sin about 0 (truncation error < 1e-8 for
// 0 <= y <= pi/2).
__device__ __forceinline__ void cutoff(float r, float rc, float k, float& fc, float& dfc) {
  const float y = r * k, y2 = y * y;
  float c = fmaf(y2, 1.0f / 479001600.0f, -1.0f / 3628800.0f);
  c = fmaf(y2, c, 1.0f / 40320.0f);
  c = fmaf(y2, c, -1.0f / 720.0f);
  c = fmaf(y2, c, 1.0f / 24.0f);
  c = fmaf(y2, c, -0.5f);
  c = fmaf(y2, c, 1.0f);
  float s = fmaf(y2, 1.0f / 6227020800.0f, -1.0f / 39916800.0f);
  s = fmaf(y2, s, 1.0f / 362880.0f);
  s = fmaf(y2, s, -1.0f / 5040.0f);
  s = fmaf(y2, s, 1.0f / 120.0f);
  s = fmaf(y2, s, -1.0f / 6.0f);
  s = fmaf(y2, s, 1.0f);
  s *= y;
  const bool in = r < rc;
  fc = in ? c * c : 0.f;
  dfc = in ? -2.f * k * s * c : 0.f;
}

// b^zeta (zeta = 2^q) by q squarings, and b^(zeta-1) as the product of the
// intermediate powers.
template <int ZSQ>
__device__ __forceinline__ void pow_zeta(float b, int zsq, float& bz, float& bzm1) {
  float p = b, prod = 1.f;
  if (ZSQ >= 0) {
#pragma unroll
    for (int i = 0; i < (ZSQ >= 0 ? ZSQ : 0); ++i) { prod *= p; p *= p; }
  } else {
    for (int i = 0; i < zsq; ++i) { prod *= p; p *= p; }
  }
  bz = p;
  bzm1 = prod;
}

template <int ZSQ>
__device__ __forceinline__ float pow_zeta1(float b, int zsq) {
  if (ZSQ >= 0) {
#pragma unroll
    for (int i = 0; i < (ZSQ >= 0 ? ZSQ : 0); ++i) b *= b;
  } else {
    for (int i = 0; i < zsq; ++i) b *= b;
  }
  return b;
}

// Reduce-scatter of V values over the 16 lanes of each half warp (both halves
// at once): lane l of a half keeps the half's sums of values V/16*l + k in
// v[k], k < V/16.
template <int V>
__device__ __forceinline__ void hw_reduce_scatter(float (&v)[V], int hl) {
#pragma unroll
  for (int w = V / 2, bit = 8; bit >= 1; w >>= 1, bit >>= 1) {
    const bool upper = (hl & bit) != 0;
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const float keep = upper ? v[k + w] : v[k];
      const float send = upper ? v[k] : v[k + w];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
}

// Flat pair index t of block (s1, s2) -> positions (u, v) in the staged
// angular neighbours.  Off-diagonal blocks: t = q n2 + r.  Diagonal blocks
// (n atoms): each unordered pair once, as (q, q + k mod n) with k <= K for the
// first n K indices (K = (n-1)/2, or n/2 - 1 for even n), then (q, q + n/2).
//
// The quotient q = t / K comes from one multiply by mg = ceil(2^31 / K):
// for t < 2^15 and K <= 2^15 the error t (mg - 2^31 / K) / 2^31 stays below
// 1 / K, so the floor is exact.  No branches: the wrap of a diagonal block
// and its tail (even n) are selects.
struct PairMap {
  int K, nK, o1, vb, vq, n;  // off-diagonal: vq = 0, n = 0 (no wrap), nK = INT_MAX (no tail)
  unsigned mg;
};

// ceil(2^31 / K) for the list lengths K <= kMaxCapA (entry 0 holds K = 1's)
struct DivMagic {
  unsigned v[kMaxCapA + 1];
  constexpr DivMagic() : v() {
    for (int k = 0; k <= kMaxCapA; ++k) v[k] = (0x80000000u + (unsigned)(k > 0 ? k : 1) - 1u) / (unsigned)(k > 0 ? k : 1);
  }
};
__constant__ DivMagic c_div_magic = DivMagic();
__device__ __forceinline__ unsigned div_magic(int K) { return c_div_magic.v[K]; }
__device__ __forceinline__ int div_by_magic(int t, unsigned mg) {
  return (int)(((unsigned long long)(unsigned)t * mg) >> 31);
}

__device__ __forceinline__ PairMap make_map(bool diag, int n1, int n2, int o1, int o2) {
  PairMap m;
  m.o1 = o1;
  if (diag) {
    m.K = (n1 & 1) ? (n1 - 1) / 2 : n1 / 2 - 1;
    if (m.K < 0) m.K = 0;
    m.nK = n1 * m.K;
    m.vb = 1;  // v = u + 1 + r, wrapped into the block
    m.vq = 1;
    m.n = n1;
  } else {
    m.K = n2;
    m.nK = 0x7fffffff;
    m.vb = o2;  // v = o2 + r
    m.vq = 0;
    m.n = 0;
  }
  m.mg = div_magic(m.K);
  return m;
}

__device__ __forceinline__ void map_pair(const PairMap& m, int t, int& u, int& v) {
  const int q = div_by_magic(t, m.mg);
  const int r = t - q * m.K;
  const int uu = m.o1 + q;
  int vv = m.vb + r + m.vq * uu;
  vv -= vv >= m.o1 + m.n ? m.n : 0;
  const int tt = t - m.nK;
  const bool tail = tt >= 0;  // diagonal, even n: (q, q + n/2)
  u = tail ? m.o1 + tt : uu;
  v = tail ? m.o1 + tt + (m.n >> 1) : vv;
}

// 2^x (MUFU; results below the normal range flush to zero)
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ f2 f2_ex2(f2 x) {
  const float2 h = f2_split(x);
  return f2_make(ex2(h.x), ex2(h.y));
}

// image shift of a list entry's virtual-cell code
__device__ __forceinline__ float4 shift_vec(int code, const SysDesc& sd) {
  const float3 v = cell_shift(code / 9 - 1, (code / 3) % 3 - 1, code % 3 - 1, sd);
  return make_float4(v.x, v.y, v.z, 0.f);
}

// Per half-warp row bookkeeping in shared memory: counts and offsets per species.
struct RowCounts {
  int nr[kMaxS], orr[kMaxS];  // radial entries and list offset per species
  int na[kMaxS], oa[kMaxS];   // staged angular entries and staging offset per species
};

__device__ __forceinline__ void load_counts(const Workspace& ws, int S, int row, bool live, int cap_a,
                                            RowCounts* rc, int hl) {
  if (hl == 0) {
    int o = 0, oa = 0;
    for (int s = 0; s < S; ++s) {
      const int n = live ? ws.cnt_r[(size_t)row * kMaxS + s] : 0;
      int a = live ? ws.cnt_a[(size_t)row * kMaxS + s] : 0;
      a = min(a, max(0, cap_a - oa));  // never stage past the buffer
      rc->nr[s] = n;
      rc->orr[s] = o;
      rc->na[s] = a;
      rc->oa[s] = oa;
      o += n;
      oa += a;
    }
  }
}

}  // namespace

// --------------------------------------------------------------------------
// forward

template <int S, int ZSQ>
__global__ void __launch_bounds__(256, 3) k_aev_fwd(const SysDesc* __restrict__ sys, DescParams P,
                                                 Workspace ws, int mode, int tile_rows, int dyn) {
  constexpr int D = kNRad * S + kNAng * S * (S + 1) / 2;
  extern __shared__ float4 sm4[];
  const int lane = threadIdx.x & 31, hl = lane & 15, half = lane >> 4;
  const int hwb = threadIdx.x >> 4;  // half warp in block, 0..15
  const int ca = ws.cap_a, cr = ws.cap_r;
  float4* geo = sm4 + (size_t)hwb * (ca + 27 + cr);
  float4* sh = geo + ca;
  float4* rad = sh + 27;  // [cr]: displacement and r^2 of every radial neighbour
  float* fcs = reinterpret_cast<float*>(sm4 + 16 * (size_t)(ca + 27 + cr)) + (size_t)hwb * ca;
  RowCounts* rc = reinterpret_cast<RowCounts*>(reinterpret_cast<float*>(sm4 + 16 * (size_t)(ca + 27 + cr)) +
                                               16 * (size_t)ca) + hwb;
  const float kr = -P.eta_r * kLog2e, ka = -P.eta_a * kLog2e;
  const float kfr = kPi / (2.f * P.rc_r), kfa = kPi / (2.f * P.rc_a);
  // sector constants (z, z+1) in shared memory, read with volatile loads in
  // the pair loop: kept in registers they push the kernel past its register
  // budget (80 at three blocks per SM) into spills and moves
  __shared__ unsigned long long s_hcs[8];
  if (threadIdx.x < 8) {
    const int q = threadIdx.x & 3;
    s_hcs[threadIdx.x] = threadIdx.x < 4 ? f2_make(P.hcos_z[2 * q], P.hcos_z[2 * q + 1]).v
                                         : f2_make(P.hsin_z[2 * q], P.hsin_z[2 * q + 1]).v;
  }
  __syncthreads();
  const volatile unsigned long long* vhcs = s_hcs;
  const f2 half2 = f2_make(0.5f, 0.5f), kr2 = f2_make(kr, kr);
  const int rows = ws.seg[S];
  int cached_sys = -1;
  // tiles of tile_rows row pairs from the work queue
  WorkQueue wq(ws.queue + kQFwd, dyn != 0);
  int pr = wq.first() * tile_rows, tile_end = pr + tile_rows;
  for (; 2 * pr < rows;) {
    const int row = 2 * pr + half;
    const bool inrow = row < rows;
    const bool live = inrow && ws.row_atom[row] >= 0;
    // FP32 form: row-major G; tensor-core forms: only the swizzled BF16 or
    // FP8 tile copy (FP8: G / s_G with the species' calibrated step s_G)
    float* Grow = ws.G + (size_t)row * D;
    char* Gh = reinterpret_cast<char*>(ws.Gh);
    float q = 1.f;
    auto put1 = [&](int f, float v) {
      if (mode == kGFp32) Grow[f] = v;
      else if (mode == kGBf16) *reinterpret_cast<__nv_bfloat16*>(Gh + gh_offset(row, f, D)) = __float2bfloat16(v);
      else Gh[gh8_offset(row, f, D)] = (char)__nv_cvt_float_to_fp8(v * q, __NV_SATFINITE, __NV_E4M3);
    };
    auto put2 = [&](int f, float v0, float v1) {  // f even
      if (mode == kGFp32) *reinterpret_cast<float2*>(Grow + f) = make_float2(v0, v1);
      else if (mode == kGBf16)
        *reinterpret_cast<__nv_bfloat162*>(Gh + gh_offset(row, f, D)) = __floats2bfloat162_rn(v0, v1);
      else
        *reinterpret_cast<__nv_fp8x2_storage_t*>(Gh + gh8_offset(row, f, D)) =
            __nv_cvt_float2_to_fp8x2(make_float2(v0 * q, v1 * q), __NV_SATFINITE, __NV_E4M3);
    };
    if (inrow && !live) {  // padding row: zero descriptor
      for (int f = hl; f < D; f += 16) put1(f, 0.f);
    }
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
      pi = ws.pos4[row];
      if (mode == kGFp8) q = 1.f / fp8_step(ws.q8[8 * pos4_species(pi)]);
      const int sid = ws.row_info[row];
      if (sid != cached_sys) {
        const SysDesc& sd = sys[sid];
        for (int c = hl; c < 27; c += 16) sh[c] = shift_vec(c, sd);
        cached_sys = sid;
      }
    }
    load_counts(ws, S, row, live, ca, rc, hl);
    __syncwarp();
    const int* lr = ws.nbr_r + (size_t)row * ws.cap_r;
    // gather every radial neighbour once (independent loads, all in flight)
    {
      const int ntot = rc->orr[S - 1] + rc->nr[S - 1];
#pragma unroll 4
      for (int k = hl; k < ntot; k += 16) {
        if (!NNP_IN(k, cr, ws.flags)) break;
        const int e = lr[k];
        if (!(NNP_IN(nbr_row(e), rows, ws.flags) && NNP_IN(nbr_code(e), 27, ws.flags))) continue;
        const float4 pj = ws.pos4[nbr_row(e)];
        const float4 sv = sh[nbr_code(e)];
        const float dx = (pj.x - pi.x) + sv.x, dy = (pj.y - pi.y) + sv.y, dz = (pj.z - pi.z) + sv.z;
        rad[k] = make_float4(dx, dy, dz, dx * dx + dy * dy + dz * dz);
      }
    }
    __syncwarp();

    // ---------------- radial
    // BF16 / FP8 forms with evenly spaced shifts: the 16 terms from two
    // anchors (4 and 12) by the ratio of neighbouring terms (DescParams),
    // 6 exponentials instead of 16; acc2[d] then holds terms (4 + d, 12 + d),
    // d = 0..3, and acc2[3 + d] terms (4 - d, 12 - d), d = 1..4.
    const bool rec = mode != kGFp32 && P.rad_even;
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
      const int n_s = rc->nr[s], o_s = rc->orr[s];
      const int nmax = max(n_s, __shfl_xor_sync(0xffffffffu, n_s, 16));
      if (nmax == 0) {  // neither row of the warp has this species in range: no reduction
        if (live) put1(s * kNRad + hl, 0.f);
        continue;
      }
      f2 acc2[kNRad / 2];
#pragma unroll
      for (int m = 0; m < kNRad / 2; ++m) acc2[m] = f2_make(0.f, 0.f);
      for (int k0 = 0; k0 < nmax; k0 += 16) {
        const int k = k0 + hl;
        if (k < n_s) {
          const float r2 = rad[o_s + k].w;
          const float r = r2 * rsqrtf(r2);
          float fc, dfc;
          cutoff(r, P.rc_r, kfr, fc, dfc);
          const f2 f = f2_make(0.25f * fc, 0.25f * fc), rr = f2_make(r, r);
          if (rec) {
            const f2 xa = f2_add(rr, f2_make(-P.shf_r[4], -P.shf_r[12]));
            const f2 ea = f2_ex2(f2_mul(kr2, f2_mul(xa, xa)));
            const f2 gx = f2_mul(f2_make(P.rad_gk, P.rad_gk), xa);
            const f2 G = f2_ex2(gx), Gi = f2_ex2(f2_mul(gx, f2_make(-1.f, -1.f)));
            acc2[0] = f2_fma(f, ea, acc2[0]);
            f2 u = ea, w = ea;
#pragma unroll
            for (int d = 1; d <= 4; ++d) {
              const f2 c = f2_make(P.rad_c[d - 1], P.rad_c[d - 1]);
              if (d < 4) {
                u = f2_mul(f2_mul(u, G), c);
                acc2[d] = f2_fma(f, u, acc2[d]);
              }
              w = f2_mul(f2_mul(w, Gi), c);
              acc2[3 + d] = f2_fma(f, w, acc2[3 + d]);
            }
          } else {
#pragma unroll
            for (int m = 0; m < kNRad / 2; ++m) {
              const f2 x = f2_add(rr, f2_make(-P.shf_r[2 * m], -P.shf_r[2 * m + 1]));
              acc2[m] = f2_fma(f, f2_ex2(f2_mul(kr2, f2_mul(x, x))), acc2[m]);
            }
          }
        }
      }
      float acc[kNRad];
      if (rec) {
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          const float2 hu = f2_split(acc2[d]), hd = f2_split(acc2[4 + d]);
          acc[4 + d] = hu.x;
          acc[12 + d] = hu.y;
          acc[3 - d] = hd.x;
          acc[11 - d] = hd.y;
        }
      } else {
#pragma unroll
        for (int m = 0; m < kNRad / 2; ++m) {
          const float2 h = f2_split(acc2[m]);
          acc[2 * m] = h.x;
          acc[2 * m + 1] = h.y;
        }
      }
      hw_reduce_scatter<kNRad>(acc, hl);
      if (live) put1(s * kNRad + hl, acc[0]);
    }

    // ---------------- angular: stage the neighbours inside rc_a
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
      const int n_a = rc->na[s], o_r = rc->orr[s], o_a = rc->oa[s];
      for (int k = hl; k < n_a; k += 16) {
        const float4 d = rad[o_r + k];
        const float dx = d.x, dy = d.y, dz = d.z, r2 = d.w;
        const float ir = rsqrtf(r2);
        const float r = r2 * ir;
        float fc, dfc;
        cutoff(r, P.rc_a, kfa, fc, dfc);
        geo[o_a + k] = make_float4(dx * ir, dy * ir, dz * ir, r);
        fcs[o_a + k] = fc;
      }
    }
    __syncwarp();
    // one species-pair block (s1, s2) of both rows of the warp
    auto ang_block = [&](int s1, int s2) {
      const bool diag = s1 == s2;
      const int n1 = rc->na[s1], n2 = rc->na[s2];
      const int T = diag ? n1 * (n1 - 1) / 2 : n1 * n2;
      const int Tmax = max(T, __shfl_xor_sync(0xffffffffu, T, 16));
      const int f0 = kNRad * S + pair_block(S, s1, s2) * kNAng + 2 * hl;
      if (Tmax == 0) {
        if (live) put2(f0, 0.f, 0.f);
        return;
      }
      const PairMap pm = make_map(diag, n1, n2, rc->oa[s1], rc->oa[s2]);
      f2 acc2[kNAngR][kNAngZ / 2];
#pragma unroll
      for (int a = 0; a < kNAngR; ++a)
#pragma unroll
        for (int zp = 0; zp < kNAngZ / 2; ++zp) acc2[a][zp] = f2_make(0.f, 0.f);
      for (int t0 = 0; t0 < Tmax; t0 += 16) {
        const int t = t0 + hl;
        if (t < T) {
          int u, v;
          map_pair(pm, t, u, v);
          const float4 gu = geo[u], gv = geo[v];
          const float c = gu.x * gv.x + gu.y * gv.y + gu.z * gv.z;
          const float uc = 0.95f * c;
          const float s2 = fmaxf(1.f - uc * uc, 1e-12f);  // >= 0.0975: |uc| <= 0.95
          const float sn = s2 * rsqrtf(s2);
          const float fp = fcs[u] * fcs[v];
          const float rbar = 0.5f * (gu.w + gv.w);
          f2 B2[kNAngR];
#pragma unroll
          for (int a = 0; a < kNAngR; ++a) {
            const float x = rbar - P.shf_a[a];
            const float Bv = fp * ex2(ka * x * x);
            B2[a] = f2_make(Bv, Bv);
          }
          const f2 uc2 = f2_make(uc, uc), sn2 = f2_make(sn, sn);
#pragma unroll
          for (int zp = 0; zp < kNAngZ / 2; ++zp) {
            f2 hcz, hsz;
            hcz.v = vhcs[zp];
            hsz.v = vhcs[4 + zp];
            f2 bz = f2_fma(sn2, hsz, f2_fma(uc2, hcz, half2));
            if (ZSQ >= 0) {
#pragma unroll
              for (int i = 0; i < (ZSQ >= 0 ? ZSQ : 0); ++i) bz = f2_mul(bz, bz);
            } else {
              for (int i = 0; i < P.zeta_sq; ++i) bz = f2_mul(bz, bz);
            }
#pragma unroll
            for (int a = 0; a < kNAngR; ++a) acc2[a][zp] = f2_fma(B2[a], bz, acc2[a][zp]);
          }
        }
      }
      float acc[kNAng];
#pragma unroll
      for (int a = 0; a < kNAngR; ++a)
#pragma unroll
        for (int zp = 0; zp < kNAngZ / 2; ++zp) {
          const float2 h = f2_split(acc2[a][zp]);
          acc[a * kNAngZ + 2 * zp] = h.x;
          acc[a * kNAngZ + 2 * zp + 1] = h.y;
        }
      hw_reduce_scatter<kNAng>(acc, hl);
      if (live) put2(f0, 2.f * acc[0], 2.f * acc[1]);
    };
    if (S <= 2) {
#pragma unroll 1
      for (int s1 = 0; s1 < S; ++s1)
#pragma unroll 1
        for (int s2 = s1; s2 < S; ++s2) ang_block(s1, s2);
    } else {
      // wide descriptors: when only some of the elements are present, most
      // blocks of a row are empty.  The row's angular features are zeroed in
      // 16-byte pieces, then only the blocks with pairs in either row of the
      // warp are evaluated (lane b tests block b).
      if (live) {
        const int fa = kNRad * S;
        if (mode == kGFp32) {
          for (int f = fa + 4 * hl; f < D; f += 64) *reinterpret_cast<float4*>(Grow + f) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (mode == kGBf16) {
          for (int f = fa + 8 * hl; f < D; f += 128) *reinterpret_cast<uint4*>(Gh + gh_offset(row, f, D)) = make_uint4(0u, 0u, 0u, 0u);
        } else {
          for (int f = fa + 16 * hl; f < D; f += 256) *reinterpret_cast<uint4*>(Gh + gh8_offset(row, f, D)) = make_uint4(0u, 0u, 0u, 0u);
        }
      }
      __syncwarp();  // the zeros land before the blocks' values
      constexpr int NB = S * (S + 1) / 2;
      const RowCounts* rc0 = rc - half;  // the counts of the warp's two rows
#pragma unroll
      for (int b0 = 0; b0 < NB; b0 += 32) {
        const int b = b0 + lane;
        int s1 = 0, s2 = 0;
#pragma unroll
        for (int q = 0, st = 0; q < S; st += S - q, ++q)
          if (b >= st) {
            s1 = q;
            s2 = q + (b - st);
          }
        bool any = false;
        if (b < NB) {
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int n1 = rc0[hh].na[s1], n2 = rc0[hh].na[s2];
            any |= (s1 == s2 ? n1 * (n1 - 1) / 2 : n1 * n2) > 0;
          }
        }
        unsigned todo = __ballot_sync(0xffffffffu, any);
        while (todo) {  // warp-uniform
          const int bb = b0 + __ffs(todo) - 1;
          todo &= todo - 1u;
          int t1 = 0, t2 = 0;
#pragma unroll
          for (int q = 0, st = 0; q < S; st += S - q, ++q)
            if (bb >= st) {
              t1 = q;
              t2 = q + (bb - st);
            }
          ang_block(t1, t2);
        }
      }
    }
    __syncwarp();
    if (++pr >= tile_end) {  // warp-uniform
      pr = wq.next(lane) * tile_rows;
      tile_end = pr + tile_rows;
    }
  }
  queue_warp_done(wq, lane);
}

// --------------------------------------------------------------------------
// backward: dE/dG -> forces (FP64 accumulation in the caller's array)
//
// Warp per row.  (1) Radial: lanes over all radial neighbours of the row
// (every species in one flat range); each lane writes its neighbour's
// radial force into the neighbour's slot and stages the angular neighbours
// (unit vector, distance, cutoff).  (2) Angular: the neighbour pairs of all
// species-pair blocks form one flat index space walked 32 at a time.  A pair
// (u, v) of block (s1, s2) contributes -(A_u e_u + B_u e_v) to u,
// -(A_v e_v + B_v e_u) to v and the negative sum to the centre; the lane
// keeps the centre's share and writes (A_u, B_u) to entry (u, v) and
// (A_v, B_v) to entry (v, u) of a per-row matrix in shared memory.
// (3) The lane of angular neighbour m sums row m of the matrix (the partner's
// unit vector comes from the staging) and adds the result to m's slot, so no
// shared-memory atomics are needed.  (4) One FP64 add per slot and component.
//
// Pair order inside a block: diagonal blocks (n neighbours) use the
// round-robin order (l, l + k mod n), k = 1..K, then (l, l + n/2) for l < n/2
// if n is even; off-diagonal blocks with lists a (m1 entries) and b
// (m2 >= m1 entries) use the wrapped diagonals (i, i + d mod m2), d-major.
// The term is symmetric in (u, v), so either list may play u.  The eight
// angular sectors (and the sixteen radial shifts) are evaluated in pairs with
// packed FP32x2 arithmetic.

namespace {

// One species-pair block of a row's angular pairs (per-warp table in shared
// memory).  Pair tl of the block: q = tl / K (multiply by mg), u = tl - q K,
// v = u + q + vq wrapped into [0, W); diagonal blocks of even n end with
// (tl - nK, tl - nK + half).
struct PairBlock {
  int base, T;      // first flat index, pairs
  int K, W, vq;     // diagonal: K = W = n, vq = 1; off-diagonal: K = ma, W = mb, vq = 0
  int oa, ob;       // staging offsets of the lists (a: u role, b: v role)
  int nK, half;     // diagonal: n K (round-robin part), n / 2 if n is even else 0; off: INT_MAX, 0
  int wo;           // offset of the block's 32 weights in dE/dG
  unsigned mg;      // ceil(2^31 / K)
};


}  // namespace

// float4 units of one warp's shared memory; the pair matrix has rows of
// mc + 1 float2 entries (the odd stride spreads a column over the banks).
// Its capacity mc is at most kBwdMatCap angular neighbours, whatever the
// staging capacity: a row with more adds its pair forces with shared-memory
// atomics instead, so one crowded row does not cost every warp its occupancy.
constexpr int kBwdMatCap = 32;
__host__ __device__ inline int bwd_mat_cap(int cap_a) { return cap_a < kBwdMatCap ? cap_a : kBwdMatCap; }
__host__ __device__ inline size_t bwd_mat_f4(int mc) { return ((size_t)mc * (mc + 1) * 2 + 3) / 4; }
// dE/dG entries a warp keeps in shared memory: the whole row, or from five
// species on (D >= 560) only the radial blocks, the angular weights being read
// through the L1 cache (the smaller footprint keeps four blocks per SM)
__host__ __device__ constexpr bool bwd_ang_global(int S) { return S >= 5; }
__host__ __device__ constexpr int bwd_wsm_floats(int S) { return bwd_ang_global(S) ? kNRad * S : desc_len(S); }
__host__ __device__ inline size_t bwd_warp_f4(int cap_a, int cap_r, int S) {
  return 27 + 2 * (size_t)cap_a + bwd_mat_f4(bwd_mat_cap(cap_a)) + (size_t)bwd_wsm_floats(S) / 4 +
         ((size_t)3 * cap_r + 3) / 4 + ((size_t)cap_r + 3) / 4 + (sizeof(PairBlock) * (S * (S + 1) / 2) + 15) / 16;
}

template <int S, int ZSQ>
__global__ void __launch_bounds__(128, 4) k_aev_bwd(const EvalIO* __restrict__ io,
                                                    const SysDesc* __restrict__ sys, DescParams P,
                                                    Workspace ws) {
  constexpr int D = kNRad * S + kNAng * S * (S + 1) / 2;
  constexpr int NB = S * (S + 1) / 2;
  constexpr unsigned FM = 0xffffffffu;
  extern __shared__ float4 sm4[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int ca = ws.cap_a, cr = ws.cap_r;
  double* const Fout = io->forces;  // FP64 forces in input order, zeroed by k_bin
  float4* sh = sm4 + (size_t)wib * bwd_warp_f4(ca, cr, S);
  float4* geo = sh + 27;
  float4* aux = geo + ca;
  float2* mat = reinterpret_cast<float2*>(aux + ca);  // [ca][ca + 1]
  const int mc = bwd_mat_cap(ca), ms = mc + 1;
  float* wsm = reinterpret_cast<float*>(aux + ca + bwd_mat_f4(mc));
  float* fsl = wsm + bwd_wsm_floats(S);
  int* origs = reinterpret_cast<int*>(reinterpret_cast<float4*>(fsl) + (3 * cr + 3) / 4);
  PairBlock* blk = reinterpret_cast<PairBlock*>(reinterpret_cast<float4*>(origs) + (cr + 3) / 4);

  const float kr = -P.eta_r * kLog2e, ka = -P.eta_a * kLog2e;
  const float kfr = kPi / (2.f * P.rc_r), kfa = kPi / (2.f * P.rc_a);
  const float zeta = (float)(1 << P.zeta_sq);
  // sector constants in pairs (z, z+1): base = 1/2 + uc hc + sn hs,
  // d(base^zeta)/dc = 0.95 zeta base^(zeta-1) (hc - (uc/sn) hs); the factor
  // 0.95 zeta (times the angular term's 2) is applied once per pair (dcs).
  // The pairs sit in shared memory and are read with volatile loads where
  // they are used: held in 16 registers they cost the pair loop more.
  __shared__ unsigned long long s_hcs[8];
  if (threadIdx.x < 8) {
    const int q = threadIdx.x & 3;
    s_hcs[threadIdx.x] = threadIdx.x < 4 ? f2_make(P.hcos_z[2 * q], P.hcos_z[2 * q + 1]).v
                                         : f2_make(P.hsin_z[2 * q], P.hsin_z[2 * q + 1]).v;
  }
  __syncthreads();
  const volatile unsigned long long* vhcs = s_hcs;
  const f2 half2 = f2_make(0.5f, 0.5f);
  const float dcs = 1.9f * zeta;
  const int rows = ws.seg[S];
  const int wpb = blockDim.x >> 5;
  const int rstride = gridDim.x * wpb;
  int cached_sys = -1;
  // the pair matrix's diagonal stays zero (a pair joins two distinct
  // neighbours), so the row sums of step (3) need no test for it
  for (int m = lane; m < mc; m += 32) mat[m * ms + m] = make_float2(0.f, 0.f);
  // the next row's metadata, counts and first 64 list entries are loaded one
  // row ahead, so their latency hides behind the current row's arithmetic
  int p_atom = -1, p_info = 0, p_cnt = 0, p_cna = 0, p_e0 = 0, p_e1 = 0;
  float4 p_pos = make_float4(0.f, 0.f, 0.f, 0.f);
  auto prefetch = [&](int rw) {
    if (rw >= rows) return;
    p_atom = ws.row_atom[rw];
    p_pos = ws.pos4[rw];
    p_info = ws.row_info[rw];
    if (lane < S) {
      p_cnt = ws.cnt_r[(size_t)rw * kMaxS + lane];
      p_cna = ws.cnt_a[(size_t)rw * kMaxS + lane];
    }
    const int* l = ws.nbr_r + (size_t)rw * cr;
    p_e0 = lane < cr ? l[lane] : 0;
    p_e1 = lane + 32 < cr ? l[lane + 32] : 0;
  };
  prefetch(blockIdx.x * wpb + wib);
  for (int row = blockIdx.x * wpb + wib; row < rows; row += rstride) {
    const bool live_row = p_atom >= 0;
    const float4 pi = p_pos;
    const int sid = p_info;
    const int cnt_l = p_cnt, cna_l = p_cna, e0 = p_e0, e1 = p_e1;
    prefetch(row + rstride);
    if (!live_row) continue;  // padding row (warp-uniform)
    __syncwarp();  // the previous row's shared data has been read
    if (sid != cached_sys) {
      const SysDesc& sd = sys[sid];
      if (lane < 27) sh[lane] = shift_vec(lane, sd);
      cached_sys = sid;
    }
    const float4* dg = reinterpret_cast<const float4*>(ws.dEdG + (size_t)row * D);
    float4* const w4s = reinterpret_cast<float4*>(wsm);
    if (S <= 2) {  // the whole dE/dG row (a row of the two-species model uses most of it)
      for (int f = lane; f < D / 4; f += 32) w4s[f] = dg[f];
    }
    // counts per species (angular ones clamped to the staging capacity)
    int nr[S], orr[S], na[S], oa[S];
    int ntot = 0, nang = 0;
#pragma unroll
    for (int q = 0; q < S; ++q) {
      nr[q] = __shfl_sync(FM, cnt_l, q);
      orr[q] = ntot;
      ntot += nr[q];
      na[q] = min(__shfl_sync(FM, cna_l, q), max(0, ca - nang));
      oa[q] = nang;
      nang += na[q];
    }
    const bool use_mat = nang <= mc;  // warp-uniform
    // pair blocks: lane b builds block b (32 blocks per round), the blocks'
    // first flat indices by a scan of their pair counts over the lanes
    int Ttot = 0, nbe = 0;  // pairs; blocks with pairs (only those are stored, in order)
#pragma unroll
    for (int r0 = 0; r0 < NB; r0 += 32) {
      const int b = r0 + lane;
      const int nl = NB - r0 < 32 ? NB - r0 : 32;  // lanes holding a block this round
      // block b -> species pair (s1, s2), s1 <= s2, s1-major
      int s1 = 0, s2 = 0;
#pragma unroll
      for (int q = 0, st = 0; q < S; st += S - q, ++q)
        if (b >= st) {
          s1 = q;
          s2 = q + (b - st);
        }
      int n1 = 0, o1 = 0, n2 = 0, o2 = 0;
#pragma unroll
      for (int q = 0; q < S; ++q) {
        if (q == s1) {
          n1 = na[q];
          o1 = oa[q];
        }
        if (q == s2) {
          n2 = na[q];
          o2 = oa[q];
        }
      }
      PairBlock pb;
      pb.wo = kNRad * S + b * kNAng;
      if (s1 == s2) {
        const int K = (n1 & 1) ? (n1 - 1) / 2 : max(0, n1 / 2 - 1);
        pb.K = pb.W = n1;
        pb.vq = 1;
        pb.oa = pb.ob = o1;
        pb.nK = n1 * K;
        pb.half = (n1 & 1) ? 0 : n1 / 2;
        pb.T = pb.nK + pb.half;
      } else {
        const bool sw = n1 > n2;  // list a is the shorter one
        pb.K = sw ? n2 : n1;
        pb.W = sw ? n1 : n2;
        pb.vq = 0;
        pb.oa = sw ? o2 : o1;
        pb.ob = sw ? o1 : o2;
        pb.nK = 0x7fffffff;
        pb.half = 0;
        pb.T = pb.K * pb.W;
      }
      const bool mine = lane < nl;
      pb.mg = div_magic(mine ? pb.K : 0);
      const int T = mine ? pb.T : 0;
      int incl = T;
#pragma unroll
      for (int o = 1; o < nl; o <<= 1) {
        const int y = __shfl_up_sync(FM, incl, o);
        if (lane >= o) incl += y;
      }
      pb.base = Ttot + incl - T;
      const unsigned has_pairs = __ballot_sync(FM, T > 0);
      if (T > 0) blk[nbe + __popc(has_pairs & ((1u << lane) - 1u))] = pb;
      nbe += __popc(has_pairs);
      Ttot += __shfl_sync(FM, incl, nl - 1);
    }
    if (S > 2) {
      // only the dE/dG blocks the row uses: the radial blocks of the species in
      // range and the angular blocks with pairs (wide descriptors, most of
      // whose blocks are unused by one row)
      __syncwarp();  // the block table is in shared memory
      const int nr_l = __shfl_sync(FM, cnt_l, (lane >> 2) & (kMaxS - 1));
      if (lane < 4 * S && nr_l > 0) w4s[lane] = dg[lane];
      if (!bwd_ang_global(S)) {
        for (int f = lane; f < 8 * nbe; f += 32) {
          const int o = (blk[f >> 3].wo >> 2) + (f & 7);
          w4s[o] = dg[o];
        }
      }
    }
    const int* lr = ws.nbr_r + (size_t)row * cr;
    float fix = 0.f, fiy = 0.f, fiz = 0.f;  // force on the centre atom
    __syncwarp();

    // ---------------- (1) radial, and staging of the angular neighbours
    for (int k = lane; k < ntot; k += 32) {
      int s = 0, o_s = 0, na_s = na[0], oa_s = 0;
#pragma unroll
      for (int q = 1; q < S; ++q)
        if (k >= orr[q]) {
          s = q;
          o_s = orr[q];
          na_s = na[q];
          oa_s = oa[q];
        }
      if (!NNP_IN(k, cr, ws.flags)) break;
      const int e = k < 32 ? e0 : (k < 64 ? e1 : lr[k]);
      if (!(NNP_IN(nbr_row(e), rows, ws.flags) && NNP_IN(nbr_code(e), 27, ws.flags))) continue;
      const float4 pj = ws.pos4[nbr_row(e)];
      const float4 sv = sh[nbr_code(e)];
      const float dx = (pj.x - pi.x) + sv.x, dy = (pj.y - pi.y) + sv.y, dz = (pj.z - pi.z) + sv.z;
      const float r2 = dx * dx + dy * dy + dz * dz;
      const float ir = rsqrtf(r2);
      const float r = r2 * ir;
      float fc, dfc;
      cutoff(r, P.rc_r, kfr, fc, dfc);
      const float4* w4 = reinterpret_cast<const float4*>(wsm + s * kNRad);
      const f2 r2v = f2_make(r, r), kr2 = f2_make(kr, kr);
      f2 s02 = f2_make(0.f, 0.f), s12 = s02;
#pragma unroll
      for (int m4 = 0; m4 < kNRad / 4; ++m4) {
        const float4 q = w4[m4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const f2 x = f2_add(r2v, f2_make(-P.shf_r[4 * m4 + 2 * h], -P.shf_r[4 * m4 + 2 * h + 1]));
          const f2 we = f2_mul(h ? f2_make(q.z, q.w) : f2_make(q.x, q.y), f2_ex2(f2_mul(kr2, f2_mul(x, x))));
          s02 = f2_add(s02, we);
          s12 = f2_fma(we, x, s12);
        }
      }
      const float2 s0h = f2_split(s02), s1h = f2_split(s12);
      const float s0 = s0h.x + s0h.y, s1 = s1h.x + s1h.y;
      // dE_i/dr_ij divided by r_ij; dE_i/dr_j = g d, dE_i/dr_i = -g d
      const float g = 0.25f * fmaf(dfc, s0, -2.f * P.eta_r * fc * s1) * ir;
      fsl[3 * k] = -g * dx;
      fsl[3 * k + 1] = -g * dy;
      fsl[3 * k + 2] = -g * dz;
      origs[k] = pos4_orig(pj);
      fix = fmaf(g, dx, fix);
      fiy = fmaf(g, dy, fiy);
      fiz = fmaf(g, dz, fiz);
      const int kk = k - o_s;
      if (kk < na_s) {  // the first na[s] entries of a species are the angular ones
        float fca, dfca;
        cutoff(r, P.rc_a, kfa, fca, dfca);
        geo[oa_s + kk] = make_float4(dx * ir, dy * ir, dz * ir, r);
        aux[oa_s + kk] = make_float4(fca, dfca, ir, __int_as_float(k));
      }
    }
    __syncwarp();

    // ---------------- (2) angular pairs, flat over the blocks
    {
      int b = 0;
      PairBlock pb = blk[0];
      for (int t = lane; t < Ttot; t += 32) {
        while (b + 1 < nbe && t >= pb.base + pb.T) pb = blk[++b];
        const int tl = t - pb.base;
        const int q = div_by_magic(tl, pb.mg);
        int u = tl - q * pb.K;
        int v = u + q + pb.vq;
        v -= v >= pb.W ? pb.W : 0;
        const int tt = tl - pb.nK;
        if (tt >= 0) {  // select: diagonal tail (u, u + n/2)
          u = tt;
          v = tt + pb.half;
        }
        u += pb.oa;
        v += pb.ob;
        const float4 gu = geo[u], gv = geo[v], au = aux[u], av = aux[v];
        const float c = gu.x * gv.x + gu.y * gv.y + gu.z * gv.z;
        const float uc = 0.95f * c;
        const float s2q = fmaxf(1.f - uc * uc, 1e-12f);
        const float isn = rsqrtf(s2q);
        const float sn = s2q * isn;
        const float ucisn = uc * isn;
        const float rbar = 0.5f * (gu.w + gv.w);
        float Be[kNAngR], Bq[kNAngR];
#pragma unroll
        for (int a = 0; a < kNAngR; ++a) {
          const float x = rbar - P.shf_a[a];
          Be[a] = ex2(ka * x * x);
          Bq[a] = -2.f * P.eta_a * x * Be[a];
        }
        const f2 uc2 = f2_make(uc, uc), sn2 = f2_make(sn, sn), nucisn2 = f2_make(-ucisn, -ucisn);
        const float* wb = (bwd_ang_global(S) ? ws.dEdG + (size_t)row * D : wsm) + pb.wo;
        f2 X2[kNAngR], Y2[kNAngR];
#pragma unroll
        for (int zp = 0; zp < kNAngZ / 2; ++zp) {
          f2 hcz, hsz;
          hcz.v = vhcs[zp];
          hsz.v = vhcs[4 + zp];
          const f2 base = f2_fma(sn2, hsz, f2_fma(uc2, hcz, half2));
          // base^(zeta-1) and base^zeta
          f2 pw = base, pm1;
          if (ZSQ >= 1) {
            f2 prod = base;
            pw = f2_mul(base, base);
#pragma unroll
            for (int i = 1; i < (ZSQ >= 1 ? ZSQ : 1); ++i) {
              prod = f2_mul(prod, pw);
              pw = f2_mul(pw, pw);
            }
            pm1 = prod;
          } else {
            const float2 bb = f2_split(base);
            float b0z, b0m, b1z, b1m;
            pow_zeta<ZSQ>(bb.x, P.zeta_sq, b0z, b0m);
            pow_zeta<ZSQ>(bb.y, P.zeta_sq, b1z, b1m);
            pw = f2_make(b0z, b1z);
            pm1 = f2_make(b0m, b1m);
          }
          const f2 dA = f2_mul(pm1, f2_fma(nucisn2, hsz, hcz));  // d(base^zeta)/dc / (0.95 zeta)
#pragma unroll
          for (int a = 0; a < kNAngR; ++a) {
            const float4* wp = reinterpret_cast<const float4*>(wb + a * kNAngZ) + (zp >> 1);
            const float4 w4 = bwd_ang_global(S) ? __ldg(wp) : *wp;
            const f2 w2 = (zp & 1) ? f2_make(w4.z, w4.w) : f2_make(w4.x, w4.y);
            if (zp == 0) {
              X2[a] = f2_mul(w2, pw);
              Y2[a] = f2_mul(w2, dA);
            } else {
              X2[a] = f2_fma(w2, pw, X2[a]);
              Y2[a] = f2_fma(w2, dA, Y2[a]);
            }
          }
        }
        float Pv = 0.f, Qv = 0.f, Rv = 0.f;
#pragma unroll
        for (int a = 0; a < kNAngR; ++a) {
          const float2 xs = f2_split(X2[a]), ys = f2_split(Y2[a]);
          const float X = xs.x + xs.y, Y = ys.x + ys.y;
          Pv = fmaf(Be[a], X, Pv);
          Qv = fmaf(Bq[a], X, Qv);
          Rv = fmaf(Be[a], Y, Rv);
        }
        // the angular term carries a factor 2 (2 ((1 + cos)/2)^zeta)
        const float fu = au.x, fv = av.x;
        const float fuv = fu * fv;
        const float dEdru = 2.f * fmaf(au.y * fv, Pv, 0.5f * fuv * Qv);
        const float dEdrv = 2.f * fmaf(fu * av.y, Pv, 0.5f * fuv * Qv);
        const float dEdc = dcs * fuv * Rv;
        // d cos/d d_u = (e_v - c e_u)/r_u ; d cos/d d_v = (e_u - c e_v)/r_v
        const float Au = fmaf(-dEdc * c, au.z, dEdru), Bu = dEdc * au.z;
        const float Av = fmaf(-dEdc * c, av.z, dEdrv), Bv = dEdc * av.z;
        if (use_mat) {
          mat[u * ms + v] = make_float2(Au, Bu);
          mat[v * ms + u] = make_float2(Av, Bv);
        } else {  // a row beyond the matrix capacity: its neighbours' shares directly
          const int su = 3 * __float_as_int(au.w), sv = 3 * __float_as_int(av.w);
          atomicAdd(&fsl[su], -fmaf(Au, gu.x, Bu * gv.x));
          atomicAdd(&fsl[su + 1], -fmaf(Au, gu.y, Bu * gv.y));
          atomicAdd(&fsl[su + 2], -fmaf(Au, gu.z, Bu * gv.z));
          atomicAdd(&fsl[sv], -fmaf(Av, gv.x, Bv * gu.x));
          atomicAdd(&fsl[sv + 1], -fmaf(Av, gv.y, Bv * gu.y));
          atomicAdd(&fsl[sv + 2], -fmaf(Av, gv.z, Bv * gu.z));
        }
        const float ca_ = Au + Bv, cb_ = Bu + Av;  // centre: g_u + g_v = (Au + Bv) e_u + (Bu + Av) e_v
        fix += ca_ * gu.x + cb_ * gv.x;
        fiy += ca_ * gu.y + cb_ * gv.y;
        fiz += ca_ * gu.z + cb_ * gv.z;
      }
    }
    __syncwarp();

    // ---------------- (3) each angular neighbour sums its row of the pair matrix
    // (the diagonal entries are zero: no pair writes them)
    for (int m = lane; m < (use_mat ? nang : 0); m += 32) {
      const float4 gm = geo[m];
      float sa = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
      const float2* row_m = mat + m * ms;
#pragma unroll 4
      for (int p = 0; p < nang; ++p) {
        const float2 c = row_m[p];
        const float4 gp = geo[p];
        sa += c.x;
        fx = fmaf(c.y, gp.x, fx);
        fy = fmaf(c.y, gp.y, fy);
        fz = fmaf(c.y, gp.z, fz);
      }
      const int slot = __float_as_int(aux[m].w);
      fsl[3 * slot] -= fmaf(sa, gm.x, fx);
      fsl[3 * slot + 1] -= fmaf(sa, gm.y, fy);
      fsl[3 * slot + 2] -= fmaf(sa, gm.z, fz);
    }
    __syncwarp();

    // ---------------- (4) FP64 reductions of the slots' forces: lane t takes
    // component t % 3 of slot t / 3, so the lanes of one instruction cover
    // about eleven atoms' contiguous x, y, z (few L2 sectors per instruction)
    for (int t = lane; t < 3 * ntot; t += 32) {
      const int k = t / 3;
      if (!(NNP_IN(k, cr, ws.flags) && NNP_IN(origs[k], io->n_atoms, ws.flags))) continue;
      atomicAdd(Fout + 3 * (size_t)origs[k] + (t - 3 * k), (double)fsl[t]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      fix += __shfl_xor_sync(FM, fix, o);
      fiy += __shfl_xor_sync(FM, fiy, o);
      fiz += __shfl_xor_sync(FM, fiz, o);
    }
    if (lane < 3 && NNP_IN(pos4_orig(pi), io->n_atoms, ws.flags))
      atomicAdd(Fout + 3 * (size_t)pos4_orig(pi) + lane, (double)(lane == 0 ? fix : (lane == 1 ? fiy : fiz)));
  }
}

// FP32 accumulators -> the caller's FP64 forces (input order).
// --------------------------------------------------------------------------
// directional derivative: dG_i = sum_j (dG_i / dr_j) . v_j (force-matching
// gradients).  Same mapping as the forward; v is per atom in input order.
//   radial:  d term_m = 1/4 exp(-eta_r x_m^2) (-2 eta_r x_m fc + fc') dr,
//            dr = e_ij . (v_j - v_i)
//   angular: d T_az = Be_a (C_z + D_z X) + Bq_a D_z Y with
//            C_z = 2 zeta b_z^(zeta-1) dbase_z dc fc_u fc_v,  D_z = 2 b_z^zeta,
//            X = fc'_u fc_v dr_u + fc_u fc'_v dr_v,  Y = fc_u fc_v (dr_u + dr_v) / 2,
//            Bq_a = dBe_a / drbar,  dc = ((e_v - c e_u).dv_u)/r_u + ((e_u - c e_v).dv_v)/r_v.

static int warps_grid_jvp(long long rows, int nsm) {
  long long g = ((rows + 1) / 2 + 7) / 8;
  if (g > (long long)nsm * 8) g = (long long)nsm * 8;
  return (int)(g < 1 ? 1 : g);
}

template <int S, int ZSQ>
__global__ void __launch_bounds__(256) k_aev_jvp(const SysDesc* __restrict__ sys, DescParams P,
                                                 Workspace ws, const double* __restrict__ vel,
                                                 float* __restrict__ dG) {
  constexpr int D = kNRad * S + kNAng * S * (S + 1) / 2;
  extern __shared__ float4 sm4[];
  const int lane = threadIdx.x & 31, hl = lane & 15, half = lane >> 4;
  const int hwb = threadIdx.x >> 4;
  const int ca = ws.cap_a;
  // per half warp: geo[ca] (unit vector, r), aux[ca] (fc, dfc, 1/r, -), dv[ca], sh[27]
  const size_t n4 = (size_t)3 * ca + 27;
  float4* geo = sm4 + hwb * n4;
  float4* aux = geo + ca;
  float4* dvs = aux + ca;
  float4* sh = dvs + ca;
  RowCounts* rc = reinterpret_cast<RowCounts*>(sm4 + 16 * n4) + hwb;
  const float kr = -P.eta_r * kLog2e, ka = -P.eta_a * kLog2e;
  const float kfr = kPi / (2.f * P.rc_r), kfa = kPi / (2.f * P.rc_a);
  const float zeta = (float)(1 << P.zeta_sq);
  const int rows = ws.seg[S];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  int cached_sys = -1;
  for (int pr = warp; 2 * pr < rows; pr += nwarps) {
    const int row = 2 * pr + half;
    const bool inrow = row < rows;
    const bool live = inrow && ws.row_atom[row] >= 0;
    float* out = dG + (size_t)row * D;
    if (inrow && !live)
      for (int f = hl; f < D; f += 16) out[f] = 0.f;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    float vix = 0.f, viy = 0.f, viz = 0.f;
    if (live) {
      pi = ws.pos4[row];
      const int oi = pos4_orig(pi);
      vix = (float)vel[3 * oi];
      viy = (float)vel[3 * oi + 1];
      viz = (float)vel[3 * oi + 2];
      const int sid = ws.row_info[row];
      if (sid != cached_sys) {
        const SysDesc& sd = sys[sid];
        for (int c = hl; c < 27; c += 16) sh[c] = shift_vec(c, sd);
        cached_sys = sid;
      }
    }
    load_counts(ws, S, row, live, ca, rc, hl);
    __syncwarp();
    const int* lr = ws.nbr_r + (size_t)row * ws.cap_r;

    // ---------------- radial
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
      const int n_s = rc->nr[s], o_s = rc->orr[s];
      const int nmax = max(n_s, __shfl_xor_sync(0xffffffffu, n_s, 16));
      float acc[kNRad];
#pragma unroll
      for (int m = 0; m < kNRad; ++m) acc[m] = 0.f;
      for (int k0 = 0; k0 < nmax; k0 += 16) {
        const int k = k0 + hl;
        if (k < n_s) {
          const int e = lr[o_s + k];
          if (!(NNP_IN(nbr_row(e), rows, ws.flags) && NNP_IN(nbr_code(e), 27, ws.flags))) continue;
          const float4 pj = ws.pos4[nbr_row(e)];
          const float4 sv = sh[nbr_code(e)];
          const float dx = (pj.x - pi.x) + sv.x, dy = (pj.y - pi.y) + sv.y, dz = (pj.z - pi.z) + sv.z;
          const float r2 = dx * dx + dy * dy + dz * dz;
          const float ir = rsqrtf(r2);
          const float r = r2 * ir;
          const int oj = pos4_orig(pj);
          const float dr = ((float)vel[3 * oj] - vix) * dx * ir + ((float)vel[3 * oj + 1] - viy) * dy * ir +
                           ((float)vel[3 * oj + 2] - viz) * dz * ir;
          float fc, dfc;
          cutoff(r, P.rc_r, kfr, fc, dfc);
#pragma unroll
          for (int m = 0; m < kNRad; ++m) {
            const float x = r - P.shf_r[m];
            const float em = exp2f(kr * x * x);
            acc[m] = fmaf(0.25f * em * fmaf(-2.f * P.eta_r * x, fc, dfc), dr, acc[m]);
          }
        }
      }
      hw_reduce_scatter<kNRad>(acc, hl);
      if (live) out[s * kNRad + hl] = acc[0];
    }

    // ---------------- angular: stage geometry and relative displacements
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
      const int n_a = rc->na[s], o_r = rc->orr[s], o_a = rc->oa[s];
      for (int k = hl; k < n_a; k += 16) {
        const int e = lr[o_r + k];
        if (!(NNP_IN(nbr_row(e), rows, ws.flags) && NNP_IN(nbr_code(e), 27, ws.flags))) continue;
        const float4 pj = ws.pos4[nbr_row(e)];
        const float4 sv = sh[nbr_code(e)];
        const float dx = (pj.x - pi.x) + sv.x, dy = (pj.y - pi.y) + sv.y, dz = (pj.z - pi.z) + sv.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float ir = rsqrtf(r2);
        const float r = r2 * ir;
        float fc, dfc;
        cutoff(r, P.rc_a, kfa, fc, dfc);
        const int oj = pos4_orig(pj);
        geo[o_a + k] = make_float4(dx * ir, dy * ir, dz * ir, r);
        aux[o_a + k] = make_float4(fc, dfc, ir, 0.f);
        dvs[o_a + k] = make_float4((float)vel[3 * oj] - vix, (float)vel[3 * oj + 1] - viy,
                                   (float)vel[3 * oj + 2] - viz, 0.f);
      }
    }
    __syncwarp();
#pragma unroll 1
    for (int s1 = 0; s1 < S; ++s1) {
#pragma unroll 1
      for (int s2 = s1; s2 < S; ++s2) {
        const bool diag = s1 == s2;
        const int n1 = rc->na[s1], n2 = rc->na[s2];
        const int T = diag ? n1 * (n1 - 1) / 2 : n1 * n2;
        const int Tmax = max(T, __shfl_xor_sync(0xffffffffu, T, 16));
        const int f0 = kNRad * S + pair_block(S, s1, s2) * kNAng + 2 * hl;
        if (Tmax == 0) {
          if (live) *reinterpret_cast<float2*>(out + f0) = make_float2(0.f, 0.f);
          continue;
        }
        const PairMap pm = make_map(diag, n1, n2, rc->oa[s1], rc->oa[s2]);
        float acc[kNAng];
#pragma unroll
        for (int q = 0; q < kNAng; ++q) acc[q] = 0.f;
        for (int t0 = 0; t0 < Tmax; t0 += 16) {
          const int t = t0 + hl;
          if (t < T) {
            int u, v;
            map_pair(pm, t, u, v);
            const float4 gu = geo[u], gv = geo[v], au = aux[u], av = aux[v], du = dvs[u], dv = dvs[v];
            const float c = gu.x * gv.x + gu.y * gv.y + gu.z * gv.z;
            const float uc = 0.95f * c;
            const float s2q = fmaxf(1.f - uc * uc, 1e-12f);
            const float isn = rsqrtf(s2q);
            const float sn = s2q * isn;
            const float ucisn = uc * isn;
            const float rbar = 0.5f * (gu.w + gv.w);
            const float dru = gu.x * du.x + gu.y * du.y + gu.z * du.z;
            const float drv = gv.x * dv.x + gv.y * dv.y + gv.z * dv.z;
            const float dcv = ((gv.x - c * gu.x) * du.x + (gv.y - c * gu.y) * du.y + (gv.z - c * gu.z) * du.z) * au.z +
                              ((gu.x - c * gv.x) * dv.x + (gu.y - c * gv.y) * dv.y + (gu.z - c * gv.z) * dv.z) * av.z;
            const float fuv = au.x * av.x;
            const float X = au.y * av.x * dru + au.x * av.y * drv;
            const float Y = 0.5f * fuv * (dru + drv);
            float Be[kNAngR], Bq[kNAngR];
#pragma unroll
            for (int a = 0; a < kNAngR; ++a) {
              const float x = rbar - P.shf_a[a];
              Be[a] = exp2f(ka * x * x);
              Bq[a] = -2.f * P.eta_a * x * Be[a];
            }
#pragma unroll
            for (int z = 0; z < kNAngZ; ++z) {
              const float base = fmaf(sn, P.hsin_z[z], fmaf(uc, P.hcos_z[z], 0.5f));
              float bz, bzm1;
              pow_zeta<ZSQ>(base, P.zeta_sq, bz, bzm1);
              const float dbase = 0.95f * fmaf(-ucisn, P.hsin_z[z], P.hcos_z[z]);
              const float Cz = 2.f * zeta * bzm1 * dbase * dcv * fuv;
              const float Dz = 2.f * bz;
              const float CDX = fmaf(Dz, X, Cz), DY = Dz * Y;
#pragma unroll
              for (int a = 0; a < kNAngR; ++a)
                acc[a * kNAngZ + z] = fmaf(Be[a], CDX, fmaf(Bq[a], DY, acc[a * kNAngZ + z]));
            }
          }
        }
        hw_reduce_scatter<kNAng>(acc, hl);
        if (live) *reinterpret_cast<float2*>(out + f0) = make_float2(acc[0], acc[1]);
      }
    }
    __syncwarp();
  }
}

size_t aev_jvp_smem(int cap_a) {
  return 16 * ((size_t)(3 * cap_a + 27) * sizeof(float4) + sizeof(RowCounts));
}

template <int S, int ZSQ>
static void jvp_t(long long rows, int nsm, cudaStream_t st, const SysDesc* sys, const DescParams& P,
                  const Workspace& ws, const double* v, float* dG) {
  k_aev_jvp<S, ZSQ><<<warps_grid_jvp(rows, nsm), 256, aev_jvp_smem(ws.cap_a), st>>>(sys, P, ws, v, dG);
}

// --------------------------------------------------------------------------
// launchers

size_t aev_fwd_smem(int cap_a, int cap_r) {
  return 16 * ((size_t)(cap_a + 27 + cap_r) * sizeof(float4) + (size_t)cap_a * sizeof(float) + sizeof(RowCounts));
}
size_t aev_bwd_smem(int cap_a, int cap_r, int S) {
  return (size_t)kBwdWarps * bwd_warp_f4(cap_a, cap_r, S) * sizeof(float4);
}

// Persistent grids: no more blocks than the work needs (items of tile rows
// per warp), capped at per_sm blocks per SM; the warps draw their tiles from
// the stage's work queue.
static int queue_grid(long long items, int warps_per_block, int nsm, int per_sm) {
  long long g = (items + warps_per_block - 1) / warps_per_block;
  const long long cap = (long long)nsm * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// tile > 0: dynamic (work queue) with tiles of that many items; tile < 0:
// static order with tiles of -tile items; 0: the default
template <int S, int ZSQ>
static void fwd_t(long long rows, int nsm, cudaStream_t st, const SysDesc* sys, const DescParams& P,
                  const Workspace& ws, int mode, int per_sm, int tile) {
  const int t = tile < 0 ? -tile : tile;
  const long long items = ((rows + 1) / 2 + t - 1) / t;
  k_aev_fwd<S, ZSQ><<<queue_grid(items, 8, nsm, per_sm), 256, aev_fwd_smem(ws.cap_a, ws.cap_r), st>>>(
      sys, P, ws, mode, t, tile > 0 ? 1 : 0);
}
// The descriptor backward keeps static order, one row per warp and step (a
// queue measured no faster for it, and its extra code cost 3%).
template <int S, int ZSQ>
static void bwd_t(long long rows, int nsm, cudaStream_t st, const EvalIO* io, const SysDesc* sys,
                  const DescParams& P, const Workspace& ws, int per_sm, int /*tile*/) {
  k_aev_bwd<S, ZSQ><<<queue_grid(rows, kBwdWarps, nsm, per_sm), 32 * kBwdWarps,
                      aev_bwd_smem(ws.cap_a, ws.cap_r, S), st>>>(io, sys, P, ws);
}

void launch_aev_fwd(long long rows, int nsm, cudaStream_t st, const SysDesc* sys, const DescParams& P,
                    const Workspace& ws, int mode, int per_sm, int tile) {
  per_sm = per_sm > 0 ? per_sm : 8;
  tile = tile != 0 ? tile : -1;
  const bool z5 = P.zeta_sq == 5;
#define FWD(s) z5 ? fwd_t<s, 5>(rows, nsm, st, sys, P, ws, mode, per_sm, tile) \
                  : fwd_t<s, -1>(rows, nsm, st, sys, P, ws, mode, per_sm, tile)
  switch (P.S) { NNP_SPECIES_CASES(FWD) }
#undef FWD
}

void launch_aev_bwd(long long rows, int nsm, cudaStream_t st, const EvalIO* io, const SysDesc* sys,
                    const DescParams& P, const Workspace& ws, int per_sm, int tile) {
  per_sm = per_sm > 0 ? per_sm : 16;
  tile = tile != 0 ? tile : -1;
  const bool z5 = P.zeta_sq == 5;
#define BWD(s) z5 ? bwd_t<s, 5>(rows, nsm, st, io, sys, P, ws, per_sm, tile) \
                  : bwd_t<s, -1>(rows, nsm, st, io, sys, P, ws, per_sm, tile)
  switch (P.S) { NNP_SPECIES_CASES(BWD) }
#undef BWD
}

template <class K>
static cudaError_t big_smem(K k) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

void launch_aev_jvp(long long rows, int nsm, cudaStream_t st, const SysDesc* sys, const DescParams& P,
                    const Workspace& ws, const double* v, float* dG) {
  const bool z5 = P.zeta_sq == 5;
#define JVP(s) z5 ? jvp_t<s, 5>(rows, nsm, st, sys, P, ws, v, dG) : jvp_t<s, -1>(rows, nsm, st, sys, P, ws, v, dG)
  switch (P.S) { NNP_SPECIES_CASES(JVP) }
#undef JVP
}

cudaError_t aev_set_smem_limits() {
  cudaError_t e = cudaSuccess;
#define BS(k) if ((e = big_smem(k)) != cudaSuccess) return e
#define FB(s) BS((k_aev_fwd<s, 5>)); BS((k_aev_fwd<s, -1>)); BS((k_aev_bwd<s, 5>)); BS((k_aev_bwd<s, -1>))
  FB(1); FB(2); FB(3); FB(4); FB(5); FB(6); FB(7); FB(8);
#define JB(s) BS((k_aev_jvp<s, 5>)); BS((k_aev_jvp<s, -1>))
  JB(1); JB(2); JB(3); JB(4); JB(5); JB(6); JB(7); JB(8);
#undef JB
#undef FB
#undef BS
  return e;
}

}  // namespace nnp
