// k_aev.cu -- ANI atomic environment vectors (radial + angular symmetry
// functions with cosine cutoffs) and their position derivatives.
//
//   radial:  G_i[s_j*16 + m] += 1/4 exp(-eta_r (r_ij - R_m)^2) fc(r_ij; rc_r)
//   angular: G_i[16S + p(s_j,s_k)*32 + a*8 + z] +=
//              2 ((1 + cos(theta' - theta_z)) / 2)^zeta
//              * exp(-eta_a ((r_ij + r_ik)/2 - R_a)^2) fc(r_ij; rc_a) fc(r_ik; rc_a)
//            with cos(theta' - theta_z) = u cos(theta_z) + sqrt(1 - u^2) sin(theta_z),
//            u = 0.95 cos(theta_ijk), so no arccos is evaluated.
//
// Forces follow Eq. 2 of the paper: F = -dE/dr, by the chain rule from
// dE/dG_i (the network backward) through these terms.
//
// Mapping: one warp per row (atom).  Radial: lanes over the neighbours of one
// species, 16 register accumulators, warp reduce-scatter.  Angular: the
// angular neighbours' unit vectors, distances and cutoffs are staged in
// shared memory; lanes run over the triplets of one species-pair block with
// 32 register accumulators (4 shifts x 8 sectors), then reduce-scatter so
// lane l owns feature l of the block.  All arithmetic FP32; per-atom forces
// are accumulated in FP64 (atomics into the caller's force array).
#include "nnp_internal.cuh"

namespace nnp {

struct AngGeo {
  float ex, ey, ez, r;
};

// Map a flat triplet index t of block (s1, s2) to neighbour positions
// (u, v) inside the angular list: off-diagonal blocks enumerate n1 x n2,
// diagonal blocks the n(n-1)/2 pairs u < v.
__device__ __forceinline__ void triplet_uv(int t, bool diag, int n1, int n2, int o1, int o2,
                                           int& u, int& v) {
  if (!diag) {
    const int q = t / n2;
    u = o1 + q;
    v = o2 + (t - q * n2);
  } else {
    const int n = n1;
    // row q holds pairs (q, q+1..n-1); first index of row q: q(2n - q - 1)/2
    float disc = (float)((2 * n - 1) * (2 * n - 1) - 8 * t);
    int q = (int)floorf(0.5f * ((float)(2 * n - 1) - sqrtf(fmaxf(disc, 0.f))));
    q = max(0, min(q, n - 2));
    while (q > 0 && q * (2 * n - q - 1) / 2 > t) --q;
    while (q + 1 <= n - 2 && (q + 1) * (2 * n - q - 2) / 2 <= t) ++q;
    const int first = q * (2 * n - q - 1) / 2;
    u = o1 + q;
    v = o1 + q + 1 + (t - first);
  }
}

__device__ __forceinline__ float pow2k(float b, int k) {
  for (int i = 0; i < k; ++i) b *= b;
  return b;
}

// Stage the angular neighbours of one row (geometry + cutoff) in shared memory.
__device__ __forceinline__ int stage_angular(const Workspace& ws, const DescParams& P, int row,
                                             float4 pi, const float ell[3], AngGeo* geo,
                                             float* fcs, float* dfcs, int* origs, int lane,
                                             int (&na_s)[kMaxS], int (&oa_s)[kMaxS]) {
  int na = 0;
#pragma unroll
  for (int s = 0; s < kMaxS; ++s) {
    na_s[s] = s < P.S ? ws.cnt_a[(size_t)row * kMaxS + s] : 0;
    oa_s[s] = na;
    na += na_s[s];
  }
  const int* la = ws.nbr_a + (size_t)row * ws.cap_a;
  for (int k = lane; k < na; k += 32) {
    const int e = la[k];
    const float4 pj = ws.pos4[nbr_row(e)];
    const float3 sh = image_shift(nbr_code(e), ell);
    const float dx = (pj.x - pi.x) + sh.x, dy = (pj.y - pi.y) + sh.y, dz = (pj.z - pi.z) + sh.z;
    const float r = sqrtf(dx * dx + dy * dy + dz * dz);
    const float ir = 1.0f / r;
    geo[k] = AngGeo{dx * ir, dy * ir, dz * ir, r};
    fcs[k] = cutoff_fc(r, P.rc_a);
    if (dfcs) dfcs[k] = cutoff_dfc(r, P.rc_a);
    if (origs) origs[k] = pos4_orig(pj);
  }
  __syncwarp();
  return na;
}

// --------------------------------------------------------------------------
// forward

template <int S>
__global__ void __launch_bounds__(256) k_aev_fwd(const SysDesc* __restrict__ sys, DescParams P,
                                                 Workspace ws, int write_bf16) {
  constexpr int D = kNRad * S + kNAng * S * (S + 1) / 2;
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  AngGeo* geo = reinterpret_cast<AngGeo*>(smem_raw) + (size_t)w * ws.cap_a;
  float* fcs = reinterpret_cast<float*>(reinterpret_cast<AngGeo*>(smem_raw) + 8 * (size_t)ws.cap_a) +
               (size_t)w * ws.cap_a;
  const int rows = ws.seg[S];
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows;
       row += (gridDim.x * blockDim.x) >> 5) {
    float* Grow = ws.G + (size_t)row * D;
    __nv_bfloat16* Ghrow = ws.Gh + (size_t)row * D;
    if (ws.row_atom[row] < 0) {
      for (int f = lane; f < D; f += 32) {
        Grow[f] = 0.f;
        if (write_bf16) Ghrow[f] = __float2bfloat16(0.f);
      }
      continue;
    }
    const float4 pi = ws.pos4[row];
    const SysDesc& sd = sys[ws.row_info[row]];
    const float ell[3] = {sd.ellf[0], sd.ellf[1], sd.ellf[2]};

    // ---------------- radial
    const int* lr = ws.nbr_r + (size_t)row * ws.cap_r;
    int o = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int n_s = ws.cnt_r[(size_t)row * kMaxS + s];
      float acc[kNRad];
#pragma unroll
      for (int m = 0; m < kNRad; ++m) acc[m] = 0.f;
      for (int k = lane; k < n_s; k += 32) {
        const int e = lr[o + k];
        const float4 pj = ws.pos4[nbr_row(e)];
        const float3 sh = image_shift(nbr_code(e), ell);
        const float dx = (pj.x - pi.x) + sh.x, dy = (pj.y - pi.y) + sh.y, dz = (pj.z - pi.z) + sh.z;
        const float r = sqrtf(dx * dx + dy * dy + dz * dz);
        const float f = 0.25f * cutoff_fc(r, P.rc_r);
#pragma unroll
        for (int m = 0; m < kNRad; ++m) {
          const float x = r - P.shf_r[m];
          acc[m] = fmaf(f, expf(-P.eta_r * x * x), acc[m]);
        }
      }
      o += n_s;
      const float val = warp_reduce_scatter<kNRad>(acc, lane);
      if ((lane & 1) == 0) {
        Grow[s * kNRad + (lane >> 1)] = val;
        if (write_bf16) Ghrow[s * kNRad + (lane >> 1)] = __float2bfloat16(val);
      }
    }

    // ---------------- angular
    int na_s[kMaxS], oa_s[kMaxS];
    stage_angular(ws, P, row, pi, ell, geo, fcs, nullptr, nullptr, lane, na_s, oa_s);
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1) {
#pragma unroll
      for (int s2 = s1; s2 < S; ++s2) {
        const int pblk = pair_block(S, s1, s2);
        const bool diag = s1 == s2;
        const int n1 = na_s[s1], n2 = na_s[s2];
        const int T = diag ? n1 * (n1 - 1) / 2 : n1 * n2;
        float acc[kNAng];
#pragma unroll
        for (int q = 0; q < kNAng; ++q) acc[q] = 0.f;
        for (int t = lane; t < T; t += 32) {
          int u, v;
          triplet_uv(t, diag, n1, n2, oa_s[s1], oa_s[s2], u, v);
          const AngGeo gu = geo[u], gv = geo[v];
          const float c = gu.ex * gv.ex + gu.ey * gv.ey + gu.ez * gv.ez;
          const float uc = 0.95f * c;
          const float sn = sqrtf(fmaxf(0.f, 1.f - uc * uc));
          const float rbar = 0.5f * (gu.r + gv.r);
          const float fp = fcs[u] * fcs[v];
          float B[kNAngR];
#pragma unroll
          for (int a = 0; a < kNAngR; ++a) {
            const float x = rbar - P.shf_a[a];
            B[a] = fp * expf(-P.eta_a * x * x);
          }
#pragma unroll
          for (int z = 0; z < kNAngZ; ++z) {
            const float base = 0.5f + uc * P.hcos_z[z] + sn * P.hsin_z[z];
            const float A = pow2k(base, P.zeta_sq);
#pragma unroll
            for (int a = 0; a < kNAngR; ++a) acc[a * kNAngZ + z] = fmaf(A, B[a], acc[a * kNAngZ + z]);
          }
        }
        float val = 0.f;
        if (__any_sync(0xffffffffu, T > 0)) val = 2.0f * warp_reduce_scatter<kNAng>(acc, lane);
        const int f = kNRad * S + pblk * kNAng + lane;
        Grow[f] = val;
        if (write_bf16) Ghrow[f] = __float2bfloat16(val);
      }
    }
    __syncwarp();
  }
}

// --------------------------------------------------------------------------
// backward: dE/dG -> forces (FP64 accumulation)

template <int S>
__global__ void __launch_bounds__(256) k_aev_bwd(const EvalIO* __restrict__ io,
                                                 const SysDesc* __restrict__ sys, DescParams P,
                                                 Workspace ws) {
  constexpr int D = kNRad * S + kNAng * S * (S + 1) / 2;
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ca = ws.cap_a;
  // per warp: geo[ca], fc[ca], dfc[ca], orig[ca], force slots[3*ca], dEdG[D]
  unsigned char* base = smem_raw + (size_t)w * (ca * (sizeof(AngGeo) + 6 * sizeof(float)) + D * sizeof(float));
  AngGeo* geo = reinterpret_cast<AngGeo*>(base);
  float* fcs = reinterpret_cast<float*>(geo + ca);
  float* dfcs = fcs + ca;
  int* origs = reinterpret_cast<int*>(dfcs + ca);
  float* fsl = reinterpret_cast<float*>(origs + ca);
  float* wsm = fsl + 3 * ca;
  double* F = io->forces;
  const int rows = ws.seg[S];
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows;
       row += (gridDim.x * blockDim.x) >> 5) {
    if (ws.row_atom[row] < 0) continue;
    const float4 pi = ws.pos4[row];
    const SysDesc& sd = sys[ws.row_info[row]];
    const float ell[3] = {sd.ellf[0], sd.ellf[1], sd.ellf[2]};
    const float* dg = ws.dEdG + (size_t)row * D;
    for (int f = lane; f < D; f += 32) wsm[f] = dg[f];
    __syncwarp();
    float fix = 0.f, fiy = 0.f, fiz = 0.f;  // force on the centre atom

    // ---------------- radial
    const int* lr = ws.nbr_r + (size_t)row * ws.cap_r;
    int o = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int n_s = ws.cnt_r[(size_t)row * kMaxS + s];
      for (int k = lane; k < n_s; k += 32) {
        const int e = lr[o + k];
        const float4 pj = ws.pos4[nbr_row(e)];
        const float3 sh = image_shift(nbr_code(e), ell);
        const float dx = (pj.x - pi.x) + sh.x, dy = (pj.y - pi.y) + sh.y, dz = (pj.z - pi.z) + sh.z;
        const float r = sqrtf(dx * dx + dy * dy + dz * dz);
        const float fc = cutoff_fc(r, P.rc_r), dfc = cutoff_dfc(r, P.rc_r);
        float g = 0.f;  // dE_i / dr
#pragma unroll
        for (int m = 0; m < kNRad; ++m) {
          const float x = r - P.shf_r[m];
          const float em = expf(-P.eta_r * x * x);
          g = fmaf(wsm[s * kNRad + m] * em, fmaf(-2.f * P.eta_r * x, fc, dfc), g);
        }
        g *= 0.25f / r;
        // dE_i/dr_j = g d, dE_i/dr_i = -g d; F = -dE/dr
        const int oj = pos4_orig(pj);
        atomicAdd(&F[3 * oj], (double)(-g * dx));
        atomicAdd(&F[3 * oj + 1], (double)(-g * dy));
        atomicAdd(&F[3 * oj + 2], (double)(-g * dz));
        fix += g * dx; fiy += g * dy; fiz += g * dz;
      }
      o += n_s;
    }

    // ---------------- angular
    int na_s[kMaxS], oa_s[kMaxS];
    const int na = stage_angular(ws, P, row, pi, ell, geo, fcs, dfcs, origs, lane, na_s, oa_s);
    for (int k = lane; k < 3 * na; k += 32) fsl[k] = 0.f;
    __syncwarp();
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1) {
#pragma unroll
      for (int s2 = s1; s2 < S; ++s2) {
        const int pblk = pair_block(S, s1, s2);
        const bool diag = s1 == s2;
        const int n1 = na_s[s1], n2 = na_s[s2];
        const int T = diag ? n1 * (n1 - 1) / 2 : n1 * n2;
        if (T == 0) continue;
        const float* wb = wsm + kNRad * S + pblk * kNAng;
        for (int t = lane; t < T; t += 32) {
          int u, v;
          triplet_uv(t, diag, n1, n2, oa_s[s1], oa_s[s2], u, v);
          const AngGeo gu = geo[u], gv = geo[v];
          const float c = gu.ex * gv.ex + gu.ey * gv.ey + gu.ez * gv.ez;
          const float uc = 0.95f * c;
          const float sn = sqrtf(fmaxf(0.f, 1.f - uc * uc));
          const float isn = 1.0f / sn;
          const float rbar = 0.5f * (gu.r + gv.r);
          float Be[kNAngR], Bq[kNAngR];
#pragma unroll
          for (int a = 0; a < kNAngR; ++a) {
            const float x = rbar - P.shf_a[a];
            Be[a] = expf(-P.eta_a * x * x);
            Bq[a] = -2.f * P.eta_a * x * Be[a];
          }
          float Pv = 0.f, Qv = 0.f, Rv = 0.f;
          const float zeta = (float)(1 << P.zeta_sq);
#pragma unroll
          for (int z = 0; z < kNAngZ; ++z) {
            const float bz = 0.5f + uc * P.hcos_z[z] + sn * P.hsin_z[z];
            const float bzm = pow2k(bz, P.zeta_sq) / bz;  // bz^(zeta-1), bz >= 0.19 here
            const float A = 2.f * bzm * bz;
            const float dA = 2.f * zeta * bzm * 0.95f * (P.hcos_z[z] - uc * P.hsin_z[z] * isn);
            float Wz = 0.f, Wq = 0.f;
#pragma unroll
            for (int a = 0; a < kNAngR; ++a) {
              const float wt = wb[a * kNAngZ + z];
              Wz = fmaf(wt, Be[a], Wz);
              Wq = fmaf(wt, Bq[a], Wq);
            }
            Pv = fmaf(A, Wz, Pv);
            Qv = fmaf(A, Wq, Qv);
            Rv = fmaf(dA, Wz, Rv);
          }
          const float fu = fcs[u], fv = fcs[v];
          const float dEdru = dfcs[u] * fv * Pv + 0.5f * fu * fv * Qv;
          const float dEdrv = fu * dfcs[v] * Pv + 0.5f * fu * fv * Qv;
          const float dEdc = fu * fv * Rv;
          const float iru = 1.f / gu.r, irv = 1.f / gv.r;
          // dc/dd_u = (e_v - c e_u)/r_u ; dc/dd_v = (e_u - c e_v)/r_v
          const float gux = dEdru * gu.ex + dEdc * (gv.ex - c * gu.ex) * iru;
          const float guy = dEdru * gu.ey + dEdc * (gv.ey - c * gu.ey) * iru;
          const float guz = dEdru * gu.ez + dEdc * (gv.ez - c * gu.ez) * iru;
          const float gvx = dEdrv * gv.ex + dEdc * (gu.ex - c * gv.ex) * irv;
          const float gvy = dEdrv * gv.ey + dEdc * (gu.ey - c * gv.ey) * irv;
          const float gvz = dEdrv * gv.ez + dEdc * (gu.ez - c * gv.ez) * irv;
          atomicAdd(&fsl[3 * u], -gux);
          atomicAdd(&fsl[3 * u + 1], -guy);
          atomicAdd(&fsl[3 * u + 2], -guz);
          atomicAdd(&fsl[3 * v], -gvx);
          atomicAdd(&fsl[3 * v + 1], -gvy);
          atomicAdd(&fsl[3 * v + 2], -gvz);
          fix += gux + gvx; fiy += guy + gvy; fiz += guz + gvz;
        }
      }
    }
    __syncwarp();
    for (int k = lane; k < na; k += 32) {
      const int oj = origs[k];
      atomicAdd(&F[3 * oj], (double)fsl[3 * k]);
      atomicAdd(&F[3 * oj + 1], (double)fsl[3 * k + 1]);
      atomicAdd(&F[3 * oj + 2], (double)fsl[3 * k + 2]);
    }
    fix = warp_sum(fix); fiy = warp_sum(fiy); fiz = warp_sum(fiz);
    if (lane == 0) {
      const int oi = pos4_orig(pi);
      atomicAdd(&F[3 * oi], (double)fix);
      atomicAdd(&F[3 * oi + 1], (double)fiy);
      atomicAdd(&F[3 * oi + 2], (double)fiz);
    }
    __syncwarp();
  }
}

size_t aev_fwd_smem(int cap_a) { return 8 * (size_t)cap_a * (sizeof(AngGeo) + sizeof(float)); }
size_t aev_bwd_smem(int cap_a, int D) {
  return 8 * ((size_t)cap_a * (sizeof(AngGeo) + 6 * sizeof(float)) + (size_t)D * sizeof(float));
}

template <int S>
void launch_aev_fwd_t(int grid, cudaStream_t st, const SysDesc* sys, const DescParams& P,
                      const Workspace& ws, int bf16) {
  k_aev_fwd<S><<<grid, 256, aev_fwd_smem(ws.cap_a), st>>>(sys, P, ws, bf16);
}
template <int S>
void launch_aev_bwd_t(int grid, cudaStream_t st, const EvalIO* io, const SysDesc* sys,
                      const DescParams& P, const Workspace& ws) {
  k_aev_bwd<S><<<grid, 256, aev_bwd_smem(ws.cap_a, P.D), st>>>(io, sys, P, ws);
}

void launch_aev_fwd(int grid, cudaStream_t st, const SysDesc* sys, const DescParams& P,
                    const Workspace& ws, int bf16) {
  switch (P.S) {
    case 1: launch_aev_fwd_t<1>(grid, st, sys, P, ws, bf16); break;
    case 2: launch_aev_fwd_t<2>(grid, st, sys, P, ws, bf16); break;
    case 3: launch_aev_fwd_t<3>(grid, st, sys, P, ws, bf16); break;
    default: launch_aev_fwd_t<4>(grid, st, sys, P, ws, bf16); break;
  }
}

void launch_aev_bwd(int grid, cudaStream_t st, const EvalIO* io, const SysDesc* sys,
                    const DescParams& P, const Workspace& ws) {
  switch (P.S) {
    case 1: launch_aev_bwd_t<1>(grid, st, io, sys, P, ws); break;
    case 2: launch_aev_bwd_t<2>(grid, st, io, sys, P, ws); break;
    case 3: launch_aev_bwd_t<3>(grid, st, io, sys, P, ws); break;
    default: launch_aev_bwd_t<4>(grid, st, io, sys, P, ws); break;
  }
}

cudaError_t aev_set_smem_limits() {
  cudaError_t e = cudaSuccess;
  const int big = 200 * 1024;
  e = cudaFuncSetAttribute(k_aev_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); if (e) return e;
  e = cudaFuncSetAttribute(k_aev_fwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); if (e) return e;
  e = cudaFuncSetAttribute(k_aev_fwd<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); if (e) return e;
  e = cudaFuncSetAttribute(k_aev_fwd<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); if (e) return e;
  e = cudaFuncSetAttribute(k_aev_bwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); if (e) return e;
  e = cudaFuncSetAttribute(k_aev_bwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); if (e) return e;
  e = cudaFuncSetAttribute(k_aev_bwd<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); if (e) return e;
  e = cudaFuncSetAttribute(k_aev_bwd<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e;
}

}  // namespace nnp
