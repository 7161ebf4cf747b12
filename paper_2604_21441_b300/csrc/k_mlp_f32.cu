// k_mlp_f32.cu -- per-element network, FP32 form (SIMT FFMA), fused:
// forward D -> 160 -> 128 -> 96 -> 1 with CELU, the atom energies E_i and
// their sum per system (FP64), and the backward pass to dE_i/dG_i (the first
// factor of the force chain rule, Eq. 2).
//
//   h_l = CELU(h_{l-1} W_l + b_l),  E_i = h_3 w_4 + b_4
//   g_3 = w_4 * CELU'(z_3),  g_{l-1} = (g_l W_l^T) * CELU'(z_{l-1}),
//   dE/dG = g_1 W_1^T,   CELU'(z) = 1 (z > 0), h/alpha + 1 (z <= 0)
//
// The evaluation kernel runs two CTAs of 256 threads per SM, one 64-row tile
// (one species) at a time; its layout is described above k_mlp_f32.  The
// force-matching passes (one CTA per SM) use the same layout, weight-chunk
// pipeline and thread mapping with two products per weight chunk.
#include "nnp_internal.cuh"

namespace nnp {

constexpr int kTM = 64;          // rows per tile
constexpr int kLDX = kTM + 4;    // padded leading dim of transposed activations
constexpr float kLog2eF = 1.4426950408889634f;  // log2(e)

// CELU with expf (the force-matching passes and weight-gradient staging)
__device__ __forceinline__ float celu_f(float z, float al, float inv_al) {
  return z > 0.f ? z : al * (expf(z * inv_al) - 1.f);
}
// The evaluation kernel's CELU: exp(z / alpha) as 2^(z kexp), kexp = log2(e) /
// alpha, on the MUFU unit (ex2.approx, about 2 ulp; results below the normal
// range flush to zero, which moves CELU by less than alpha 2^-126).  e gets
// exp(z / alpha), which is CELU'(z) for z <= 0.
__device__ __forceinline__ float celu_ex2(float z, float al, float kexp, float& e) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(z * kexp));
  e = y;
  return z > 0.f ? z : al * (y - 1.f);
}
// CELU'(z) from h = CELU(z): 1 for h > 0, h/alpha + 1 otherwise
__device__ __forceinline__ float dcelu_from_h(float h, float inv_al) {
  return h > 0.f ? 1.f : fmaf(h, inv_al, 1.f);
}

// ---- the evaluation kernel (k_mlp_f32) ----------------------------------
// Two CTAs of 256 threads per SM.  A 64-row tile's activations stay in shared
// memory transposed with the padded leading dimension kLDX: a thread's eight
// rows at one feature are two float4 at fixed offsets from the feature's row
// (the same address across the warp, a broadcast), and the float4 stores of an
// epilogue from eight consecutive features land on all 32 banks.  Weights
// stream through one 16-row chunk that each thread fetches into registers a
// chunk ahead, so the L2 latency hides behind the current chunk's arithmetic.
// Accumulators pair neighbouring rows for fma.rn.f32x2: every lane still
// computes each output with one FP32 fma per k, in k order.  Shared memory:
// H1T | H2T | H3T | Bs = 114,688 bytes; the first layer's staged input chunk
// lives in H2T, which is free until the second layer's epilogue.
constexpr int kNKC = 16;       // k-chunk of the streamed weights
constexpr int kNBsN = 160;     // widest product (wider dE/dG: column blocks)
constexpr int kNColBlock = 128;

// One weight chunk (and, for the first layer, one staged input chunk) in
// flight in registers: kNKC x N floats of B as float4, at most three per thread.
struct NetPf {
  float4 b[3];
  float4 a;
};

// Fetch chunk k0 of a product with N columns: B rows of ldb floats (CH: a
// column block whose columns from ncol on are absent, read as zero); STAGED:
// also the 64 x kNKC input chunk from rows of global memory (lda).
template <int N, bool CH, bool STAGED>
__device__ __forceinline__ void net_fetch(NetPf& pf, const float* __restrict__ Bg, int ldb, int ncol,
                                          const float* __restrict__ Ag, int lda, int k0) {
  constexpr int NV = kNKC * N / 4;
  constexpr int PV = (NV + 255) / 256;
  static_assert(PV <= 3, "weight chunk too wide");
  const int tid = threadIdx.x;
#pragma unroll
  for (int p = 0; p < PV; ++p) {
    const int i = tid + 256 * p;
    if (NV % 256 == 0 || i < NV) {
      const int kk = i / (N / 4), c = 4 * (i - kk * (N / 4));
      if (!CH || c < ncol)
        pf.b[p] = __ldg(reinterpret_cast<const float4*>(Bg + (size_t)(k0 + kk) * ldb + c));
      else
        pf.b[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if (STAGED) pf.a = __ldg(reinterpret_cast<const float4*>(Ag + (size_t)(tid >> 2) * lda + k0 + 4 * (tid & 3)));
}

template <int N, bool STAGED>
__device__ __forceinline__ void net_stash(const NetPf& pf, float* Bs, float* As) {
  constexpr int NV = kNKC * N / 4;
  constexpr int PV = (NV + 255) / 256;
  const int tid = threadIdx.x;
#pragma unroll
  for (int p = 0; p < PV; ++p) {
    const int i = tid + 256 * p;
    if (NV % 256 == 0 || i < NV) reinterpret_cast<float4*>(Bs)[i] = pf.b[p];
  }
  if (STAGED) {
    const int r = tid >> 2, k4 = 4 * (tid & 3);
    As[k4 * kLDX + r] = pf.a.x;
    As[(k4 + 1) * kLDX + r] = pf.a.y;
    As[(k4 + 2) * kLDX + r] = pf.a.z;
    As[(k4 + 3) * kLDX + r] = pf.a.w;
  }
}

// acc[p][j] += A(64 x K) B(K x N) for rows 8ty+2p, 8ty+2p+1 and column tx+32j.
// A: transposed activations AT[k][kLDX], or (STAGED) rows of global memory
// (lda) staged chunk by chunk in As[kNKC][kLDX].  pf holds chunk 0 on entry
// (fetched by the caller or by the previous product); during the last chunk
// next(pf) fetches the following product's chunk 0.
template <int N, bool CH, bool STAGED, class Next>
__device__ __forceinline__ void net_gemm(f2 (&acc)[4][(N + 31) / 32], const float* AT,
                                         const float* __restrict__ Ag, int lda, int K,
                                         const float* __restrict__ Bg, int ldb, int ncol, float* Bs,
                                         float* As, NetPf& pf, Next next) {
  constexpr int NJ = (N + 31) / 32;
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  const int nch = K / kNKC;
  for (int ch = 0; ch < nch; ++ch) {
    __syncthreads();  // every warp is done with the previous chunk
    net_stash<N, STAGED>(pf, Bs, As);
    __syncthreads();
    if (ch + 1 < nch)
      net_fetch<N, CH, STAGED>(pf, Bg, ldb, ncol, Ag, lda, (ch + 1) * kNKC);
    else
      next(pf);
    const float* Ab = (STAGED ? As : AT + (size_t)ch * kNKC * kLDX) + ty * 8;
#pragma unroll
    for (int kk = 0; kk < kNKC; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(Ab + kk * kLDX);
      const float4 a1 = *reinterpret_cast<const float4*>(Ab + kk * kLDX + 4);
      const f2 ap[4] = {f2_make(a0.x, a0.y), f2_make(a0.z, a0.w), f2_make(a1.x, a1.y), f2_make(a1.z, a1.w)};
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int col = tx + 32 * j;
        const float b = (N % 32 == 0 || col < N) ? Bs[kk * N + col] : 0.f;
        const f2 bb = f2_make(b, b);
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[p][j] = f2_fma(ap[p], bb, acc[p][j]);
      }
    }
  }
}

template <int N>
__device__ __forceinline__ void net_zero(f2 (&acc)[4][(N + 31) / 32]) {
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int j = 0; j < (N + 31) / 32; ++j) acc[p][j] = f2_make(0.f, 0.f);
}

// the eight values of column j, rows 8ty..8ty+7
template <int NJ>
__device__ __forceinline__ void net_col(const f2 (&acc)[4][NJ], int j, float (&v)[8]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float2 t = f2_split(acc[p][j]);
    v[2 * p] = t.x;
    v[2 * p + 1] = t.y;
  }
}

// forward epilogue: HT(col, rows) = CELU(acc + b)
template <int N>
__device__ __forceinline__ void net_store_celu(const f2 (&acc)[4][N / 32], const float* bias, float* HT,
                                               float al, float kexp) {
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < N / 32; ++j) {
    const int col = tx + 32 * j;
    const float bb = bias[col];
    float h[8];
    net_col<N / 32>(acc, j, h);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float e;
      h[i] = celu_ex2(h[i] + bb, al, kexp, e);
    }
    *reinterpret_cast<float4*>(HT + col * kLDX + ty * 8) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(HT + col * kLDX + ty * 8 + 4) = make_float4(h[4], h[5], h[6], h[7]);
  }
}

// backward epilogue: HT(col, rows) <- acc * CELU'(h), h = HT(col, rows)
template <int N>
__device__ __forceinline__ void net_store_bwd(const f2 (&acc)[4][N / 32], float* HT, float inv_al) {
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < N / 32; ++j) {
    const int col = tx + 32 * j;
    float4* p0 = reinterpret_cast<float4*>(HT + col * kLDX + ty * 8);
    float4* p1 = p0 + 1;
    const float4 h0 = *p0, h1 = *p1;
    const float h[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
    float g[8];
    net_col<N / 32>(acc, j, g);
#pragma unroll
    for (int i = 0; i < 8; ++i) g[i] *= dcelu_from_h(h[i], inv_al);
    *p0 = make_float4(g[0], g[1], g[2], g[3]);
    *p1 = make_float4(g[4], g[5], g[6], g[7]);
  }
}

// dE/dG columns [c0, c0 + ncol) of the tile's rows (acc = 1: added to what
// an earlier ensemble member left there)
template <int N>
__device__ __forceinline__ void net_store_dedg(const f2 (&acc)[4][(N + 31) / 32], float* dEdG, int D, int row0,
                                               int c0, int ncol, int add) {
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < (N + 31) / 32; ++j) {
    const int col = tx + 32 * j;
    if (col >= ncol) continue;
    float v[8];
    net_col<(N + 31) / 32>(acc, j, v);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float* o = dEdG + (size_t)(row0 + ty * 8 + i) * D + c0 + col;
      *o = add ? *o + v[i] : v[i];
    }
  }
}

// acc = 1: add E_i and dE/dG to what an earlier ensemble member left there
template <int S>
__global__ void __launch_bounds__(256, 2) k_mlp_f32(const EvalIO* __restrict__ io,
                                                    DescParams P, Workspace ws, MlpF32Weights Wt, int acc) {
  constexpr int D = kNRad * S + kNAng * S * (S + 1) / 2;
  extern __shared__ float4 smf4[];
  float* H1T = reinterpret_cast<float*>(smf4);  // [160 features][kLDX]
  float* H2T = H1T + kH1 * kLDX;                // [128][kLDX]
  float* H3T = H2T + kH2 * kLDX;                // [96][kLDX]
  float* Bs = H3T + kH3 * kLDX;                 // [kNKC][<= 160]
  float* As = H2T;                              // [kNKC][kLDX], first layer only
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
  const float al = P.celu_alpha, inv_al = 1.f / P.celu_alpha, kexp = kLog2eF * inv_al;
  const int rows = ws.seg[S];
  const int ntiles = rows / kTM;
  auto tile_species = [&](int t) {
    int s = pos4_species(ws.pos4[t * kTM]);
    return NNP_IN(s, P.S, ws.flags) ? s : 0;
  };
  // Tiles: the first by block index, the later ones from a counter (the
  // launch's last block resets it), each claimed one tile ahead so that its
  // species is known early.  Every product's first chunk is fetched during
  // the previous product's last one (the first layer of the next tile during
  // the last dE/dG block).
  __shared__ int s_claim[2];
  int* const tq = ws.queue + kQNet;  // claim counter, blocks done
  NetPf pf;
  int sp = 0, tile = blockIdx.x, ntile = ntiles;
  if (tile < ntiles) {
    if (threadIdx.x == 0) s_claim[0] = (int)gridDim.x + atomicAdd(tq, 1);
    sp = tile_species(tile);
    net_fetch<kH1, false, true>(pf, Wt.W[sp][0], kH1, kH1, ws.G + (size_t)tile * kTM * D, D, 0);
    __syncthreads();
    ntile = s_claim[0];
  }
  for (int it = 1; tile < ntiles; ++it) {
    const int row0 = tile * kTM;
    // the tile after the next one (read at the end of this one, past many barriers)
    if (threadIdx.x == 0 && ntile < ntiles) s_claim[it & 1] = (int)gridDim.x + atomicAdd(tq, 1);
    const int sp_next = ntile < ntiles ? tile_species(ntile) : 0;
    auto next_tile = [&](NetPf& q) {
      if (ntile < ntiles)
        net_fetch<kH1, false, true>(q, Wt.W[sp_next][0], kH1, kH1, ws.G + (size_t)ntile * kTM * D, D, 0);
    };
    // ---- forward
    {
      f2 a1[4][kH1 / 32];
      net_zero<kH1>(a1);
      net_gemm<kH1, false, true>(a1, nullptr, ws.G + (size_t)row0 * D, D, D, Wt.W[sp][0], kH1, kH1, Bs, As, pf,
                                 [&](NetPf& q) { net_fetch<kH2, false, false>(q, Wt.W[sp][1], kH2, kH2, nullptr, 0, 0); });
      net_store_celu<kH1>(a1, Wt.b[sp][0], H1T, al, kexp);
    }
    {
      f2 a2[4][kH2 / 32];
      net_zero<kH2>(a2);
      net_gemm<kH2, false, false>(a2, H1T, nullptr, 0, kH1, Wt.W[sp][1], kH2, kH2, Bs, As, pf,
                                  [&](NetPf& q) { net_fetch<kH3, false, false>(q, Wt.W[sp][2], kH3, kH3, nullptr, 0, 0); });
      net_store_celu<kH2>(a2, Wt.b[sp][1], H2T, al, kexp);
    }
    {
      f2 a3[4][kH3 / 32];
      net_zero<kH3>(a3);
      net_gemm<kH3, false, false>(a3, H2T, nullptr, 0, kH2, Wt.W[sp][2], kH3, kH3, Bs, As, pf,
                                  [&](NetPf& q) { net_fetch<kH2, false, false>(q, Wt.WT[sp][2], kH2, kH2, nullptr, 0, 0); });
      // layer 3 epilogue: energy and g3 = w4 * CELU'(z3), stored in H3T
      const float* w4 = Wt.W[sp][3];
      const float* b3 = Wt.b[sp][2];
      float e[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) e[i] = 0.f;
#pragma unroll
      for (int j = 0; j < kH3 / 32; ++j) {
        const int col = tx + 32 * j;
        const float ww = w4[col], bb = b3[col];
        float z[8], g[8];
        net_col<kH3 / 32>(a3, j, z);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float zz = z[i] + bb;
          float ez;
          const float h = celu_ex2(zz, al, kexp, ez);
          e[i] = fmaf(h, ww, e[i]);
          g[i] = ww * (zz > 0.f ? 1.f : ez);
        }
        *reinterpret_cast<float4*>(H3T + col * kLDX + ty * 8) = make_float4(g[0], g[1], g[2], g[3]);
        *reinterpret_cast<float4*>(H3T + col * kLDX + ty * 8 + 4) = make_float4(g[4], g[5], g[6], g[7]);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) e[i] = warp_sum(e[i]);
      // rows ty*8 .. ty*8+7 of this warp: lane i < 8 holds row ty*8 + i
      float ev = e[0];
#pragma unroll
      for (int i = 1; i < 8; ++i) ev = (tx == i) ? e[i] : ev;
      const int row = row0 + ty * 8 + (tx & 7);
      const bool valid = tx < 8 && ws.row_atom[row] >= 0;
      const int sys = ws.row_info[row];
      ev += Wt.b[sp][3][0];
      if (tx < 8) {
        const float v = valid ? ev : 0.f;
        ws.Ei[row] = acc ? ws.Ei[row] + v : v;
      }
      unsigned todo = __ballot_sync(0xffffffffu, valid);
      while (todo) {  // per-system runs: shuffle sum, one FP64 add each
        const int leader = __ffs(todo) - 1;
        const int ls = __shfl_sync(0xffffffffu, sys, leader);
        const bool mine = valid && sys == ls;
        float x = mine ? ev : 0.f;
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (tx == leader) atomicAdd(&io->energies[ls], (double)x);
        todo &= ~__ballot_sync(0xffffffffu, mine);
      }
    }
    // ---- backward (each product's first chunk barrier orders the previous
    // epilogue's stores before their reads)
    {
      f2 b2[4][kH2 / 32];
      net_zero<kH2>(b2);
      net_gemm<kH2, false, false>(b2, H3T, nullptr, 0, kH3, Wt.WT[sp][2], kH2, kH2, Bs, As, pf,
                                  [&](NetPf& q) { net_fetch<kH1, false, false>(q, Wt.WT[sp][1], kH1, kH1, nullptr, 0, 0); });
      net_store_bwd<kH2>(b2, H2T, inv_al);
    }
    {
      f2 b1[4][kH1 / 32];
      net_zero<kH1>(b1);
      net_gemm<kH1, false, false>(b1, H2T, nullptr, 0, kH2, Wt.WT[sp][1], kH1, kH1, Bs, As, pf, [&](NetPf& q) {
        if constexpr (D <= kNBsN)
          net_fetch<D, false, false>(q, Wt.WT[sp][0], D, D, nullptr, 0, 0);
        else
          net_fetch<kNColBlock, true, false>(q, Wt.WT[sp][0], D, min(kNColBlock, D), nullptr, 0, 0);
      });
      net_store_bwd<kH1>(b1, H1T, inv_al);
    }
    if constexpr (D <= kNBsN) {
      f2 g[4][(D + 31) / 32];
      net_zero<D>(g);
      net_gemm<D, false, false>(g, H1T, nullptr, 0, kH1, Wt.WT[sp][0], D, D, Bs, As, pf, next_tile);
      net_store_dedg<D>(g, ws.dEdG, D, row0, 0, D, acc);
    } else {
      for (int c0 = 0; c0 < D; c0 += kNColBlock) {
        const int nc = min(kNColBlock, D - c0);
        f2 g[4][kNColBlock / 32];
        net_zero<kNColBlock>(g);
        const int c1 = c0 + kNColBlock;
        net_gemm<kNColBlock, true, false>(g, H1T, nullptr, 0, kH1, Wt.WT[sp][0] + c0, D, nc, Bs, As, pf,
                                          [&](NetPf& q) {
                                            if (c1 < D)
                                              net_fetch<kNColBlock, true, false>(q, Wt.WT[sp][0] + c1, D,
                                                                                 min(kNColBlock, D - c1),
                                                                                 nullptr, 0, 0);
                                            else
                                              next_tile(q);
                                          });
        net_store_dedg<kNColBlock>(g, ws.dEdG, D, row0, c0, nc, acc);
      }
    }
    sp = sp_next;
    tile = ntile;
    ntile = tile < ntiles ? s_claim[it & 1] : ntiles;
  }
  if (threadIdx.x == 0) {  // after this block's last claim; the last block resets the counter
    __threadfence();
    if (atomicAdd(tq + 1, 1) == (int)gridDim.x - 1) {
      atomicExch(tq, 0);
      atomicExch(tq + 1, 0);
    }
  }
}

// --------------------------------------------------------------------------
// Force-matching weight gradients (FP32, second order).
// With v = dL/dF, dL/dtheta = -d/dtheta sum_i <dE_i/dG_i, dG_i> where dG_i is
// the directional derivative of atom i's descriptor along v (computed by the
// descriptor kernels).  Per atom, forward-over-reverse through the network:
//   tangent forward:  dz_l = dh_{l-1} W_l,  dh_l = CELU'(z_l) dz_l  (dh_0 = dG)
//   reverse of phi = dh_3 . w_4:
//     t_3 = w_4 CELU'(z_3),                 p_3 = w_4 CELU''(z_3) dz_3
//     t_l = CELU'(z_l) (t_{l+1} W_{l+1}^T),  p_l = CELU'(z_l) (p_{l+1} W_{l+1}^T) + CELU''(z_l) dz_l (t_{l+1} W_{l+1}^T)
//   dL/dW_l = -sum_i (dh_{l-1}^T t_l + h_{l-1}^T p_l),  dL/db_l = -sum_i p_l,
//   dL/dw_4 = -sum_i dh_3,  dL/db_4 = 0.
// Per-row buffers [rows][384]: z1 | z2 | z3 (160 | 128 | 96) and the same for dz, t, p.

// Two products with the same B for the force-matching passes (primal and
// tangent, or the two adjoints): acc += A B and acc2 += A2 B, one weight
// chunk stream for both, fetched a chunk ahead, row-paired f32x2 FMAs (each
// output still one FP32 fma per k, in k order).  A, A2: transposed in shared
// memory (AT, AT2 [k][kLDX]) or (STAGED) rows of global memory (Ag, Ag2, lda)
// staged in As, As2 [kNKC][kLDX].  B: rows of N floats.
template <int N, bool STAGED>
__device__ __forceinline__ void fm_gemm2(f2 (&acc)[4][N / 32], f2 (&acc2)[4][N / 32], const float* AT,
                                         const float* AT2, const float* __restrict__ Ag,
                                         const float* __restrict__ Ag2, int lda, int K,
                                         const float* __restrict__ Bg, float* Bs, float* As, float* As2) {
  constexpr int NJ = N / 32;
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  NetPf pf;
  float4 pa2 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto fetch = [&](int k0) {
    net_fetch<N, false, STAGED>(pf, Bg, N, N, Ag, lda, k0);
    if (STAGED) pa2 = __ldg(reinterpret_cast<const float4*>(Ag2 + (size_t)(tid >> 2) * lda + k0 + 4 * (tid & 3)));
  };
  const int nch = K / kNKC;
  fetch(0);
  for (int ch = 0; ch < nch; ++ch) {
    __syncthreads();
    net_stash<N, STAGED>(pf, Bs, As);
    if (STAGED) {
      const int r = tid >> 2, k4 = 4 * (tid & 3);
      As2[k4 * kLDX + r] = pa2.x;
      As2[(k4 + 1) * kLDX + r] = pa2.y;
      As2[(k4 + 2) * kLDX + r] = pa2.z;
      As2[(k4 + 3) * kLDX + r] = pa2.w;
    }
    __syncthreads();
    if (ch + 1 < nch) fetch((ch + 1) * kNKC);
    const float* Ab = (STAGED ? As : AT + (size_t)ch * kNKC * kLDX) + ty * 8;
    const float* Ab2 = (STAGED ? As2 : AT2 + (size_t)ch * kNKC * kLDX) + ty * 8;
#pragma unroll
    for (int kk = 0; kk < kNKC; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(Ab + kk * kLDX);
      const float4 a1 = *reinterpret_cast<const float4*>(Ab + kk * kLDX + 4);
      const float4 c0 = *reinterpret_cast<const float4*>(Ab2 + kk * kLDX);
      const float4 c1 = *reinterpret_cast<const float4*>(Ab2 + kk * kLDX + 4);
      const f2 ap[4] = {f2_make(a0.x, a0.y), f2_make(a0.z, a0.w), f2_make(a1.x, a1.y), f2_make(a1.z, a1.w)};
      const f2 cp[4] = {f2_make(c0.x, c0.y), f2_make(c0.z, c0.w), f2_make(c1.x, c1.y), f2_make(c1.z, c1.w)};
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const float b = Bs[kk * N + tx + 32 * j];
        const f2 bb = f2_make(b, b);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          acc[p][j] = f2_fma(ap[p], bb, acc[p][j]);
          acc2[p][j] = f2_fma(cp[p], bb, acc2[p][j]);
        }
      }
    }
  }
}

// f2 accumulators (row pairs) -> acc[row][column] for the epilogues
template <int NJ>
__device__ __forceinline__ void fm_rows(const f2 (&a)[4][NJ], float (&out)[8][NJ]) {
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    float v[8];
    net_col<NJ>(a, j, v);
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i][j] = v[i];
  }
}

constexpr int kFmW = kH1 + kH2 + kH3;  // 384
__host__ __device__ constexpr int fm_off(int layer0) {  // z1 | z2 | z3 column offsets
  return layer0 == 0 ? 0 : (layer0 == 1 ? kH1 : kH1 + kH2);
}

__device__ __forceinline__ float d2celu(float z, float inv_al) {
  return z > 0.f ? 0.f : expf(z * inv_al) * inv_al;
}

// Forward epilogue of the tangent pass: z = acc + b, dz = accd; store both rows-major
// in global buffers and h, dh transposed in shared memory.
template <int N>
__device__ __forceinline__ void fm_store_fwd(const float (&acc)[8][N / 32], const float (&accd)[8][N / 32],
                                             const float* bias, float* HT, float* DHT, float* z, float* dz,
                                             int row0, int off, float al, float inv_al) {
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < N / 32; ++j) {
    const int col = tx + 32 * j;
    const float bb = bias[col];
    float h[8], dh[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float zz = acc[i][j] + bb;
      const size_t g = (size_t)(row0 + ty * 8 + i) * kFmW + off + col;
      z[g] = zz;
      dz[g] = accd[i][j];
      h[i] = celu_f(zz, al, inv_al);
      dh[i] = dcelu_from_h(h[i], inv_al) * accd[i][j];
    }
    if (HT) {
      *reinterpret_cast<float4*>(HT + col * kLDX + ty * 8) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(HT + col * kLDX + ty * 8 + 4) = make_float4(h[4], h[5], h[6], h[7]);
      *reinterpret_cast<float4*>(DHT + col * kLDX + ty * 8) = make_float4(dh[0], dh[1], dh[2], dh[3]);
      *reinterpret_cast<float4*>(DHT + col * kLDX + ty * 8 + 4) = make_float4(dh[4], dh[5], dh[6], dh[7]);
    }
  }
}

template <int S>
__global__ void __launch_bounds__(256, 1) k_fm_fwd(DescParams P, Workspace ws, MlpF32Weights Wt,
                                                   const float* __restrict__ dG, float* z, float* dz) {
  constexpr int D = kNRad * S + kNAng * S * (S + 1) / 2;
  extern __shared__ float smf[];
  float* H1T = smf;
  float* DH1T = H1T + kH1 * kLDX;
  float* H2T = DH1T + kH1 * kLDX;
  float* DH2T = H2T + kH2 * kLDX;
  float* Bs = DH2T + kH2 * kLDX;  // [kNKC][160]: every product here has N <= 160
  float* As = Bs + kNKC * kH1;    // [kNKC][kLDX] each
  float* As2 = As + kNKC * kLDX;
  const float al = P.celu_alpha, inv_al = 1.f / P.celu_alpha;
  const int ntiles = ws.seg[S] / kTM;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int row0 = tile * kTM;
    int sp = pos4_species(ws.pos4[row0]);
    if (!NNP_IN(sp, P.S, ws.flags)) sp = 0;
    {
      f2 a[4][kH1 / 32], ad[4][kH1 / 32];
      net_zero<kH1>(a);
      net_zero<kH1>(ad);
      fm_gemm2<kH1, true>(a, ad, nullptr, nullptr, ws.G + (size_t)row0 * D, dG + (size_t)row0 * D, D, D,
                          Wt.W[sp][0], Bs, As, As2);
      float acc[8][kH1 / 32], accd[8][kH1 / 32];
      fm_rows<kH1 / 32>(a, acc);
      fm_rows<kH1 / 32>(ad, accd);
      fm_store_fwd<kH1>(acc, accd, Wt.b[sp][0], H1T, DH1T, z, dz, row0, fm_off(0), al, inv_al);
    }
    {
      f2 a[4][kH2 / 32], ad[4][kH2 / 32];
      net_zero<kH2>(a);
      net_zero<kH2>(ad);
      fm_gemm2<kH2, false>(a, ad, H1T, DH1T, nullptr, nullptr, 0, kH1, Wt.W[sp][1], Bs, As, As2);
      float acc[8][kH2 / 32], accd[8][kH2 / 32];
      fm_rows<kH2 / 32>(a, acc);
      fm_rows<kH2 / 32>(ad, accd);
      fm_store_fwd<kH2>(acc, accd, Wt.b[sp][1], H2T, DH2T, z, dz, row0, fm_off(1), al, inv_al);
    }
    {
      f2 a[4][kH3 / 32], ad[4][kH3 / 32];
      net_zero<kH3>(a);
      net_zero<kH3>(ad);
      fm_gemm2<kH3, false>(a, ad, H2T, DH2T, nullptr, nullptr, 0, kH2, Wt.W[sp][2], Bs, As, As2);
      float acc[8][kH3 / 32], accd[8][kH3 / 32];
      fm_rows<kH3 / 32>(a, acc);
      fm_rows<kH3 / 32>(ad, accd);
      fm_store_fwd<kH3>(acc, accd, Wt.b[sp][2], nullptr, nullptr, z, dz, row0, fm_off(2), al, inv_al);
    }
    __syncthreads();
  }
}

// Reverse epilogue: t = s' th, p = s' ph + s'' dz th (zero on padding rows);
// store rows-major in global buffers and transposed in shared memory.
template <int N>
__device__ __forceinline__ void fm_store_rev(const float (&th)[8][N / 32], const float (&ph)[8][N / 32],
                                             const float* z, const float* dz, float* t, float* p,
                                             float* TT, float* PT, int row0, int off,
                                             const int (&valid)[8], float inv_al) {
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < N / 32; ++j) {
    const int col = tx + 32 * j;
    float tv[8], pv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const size_t g = (size_t)(row0 + ty * 8 + i) * kFmW + off + col;
      const float zz = z[g], dd = dz[g];
      const float s1 = zz > 0.f ? 1.f : expf(zz * inv_al);
      tv[i] = valid[i] ? s1 * th[i][j] : 0.f;
      pv[i] = valid[i] ? fmaf(s1, ph[i][j], d2celu(zz, inv_al) * dd * th[i][j]) : 0.f;
      t[g] = tv[i];
      p[g] = pv[i];
    }
    if (TT) {
      *reinterpret_cast<float4*>(TT + col * kLDX + ty * 8) = make_float4(tv[0], tv[1], tv[2], tv[3]);
      *reinterpret_cast<float4*>(TT + col * kLDX + ty * 8 + 4) = make_float4(tv[4], tv[5], tv[6], tv[7]);
      *reinterpret_cast<float4*>(PT + col * kLDX + ty * 8) = make_float4(pv[0], pv[1], pv[2], pv[3]);
      *reinterpret_cast<float4*>(PT + col * kLDX + ty * 8 + 4) = make_float4(pv[4], pv[5], pv[6], pv[7]);
    }
  }
}

template <int S>
__global__ void __launch_bounds__(256, 1) k_fm_rev(DescParams P, Workspace ws, MlpF32Weights Wt,
                                                   const float* z, const float* dz, float* t, float* p) {
  extern __shared__ float smf[];
  float* T3 = smf;
  float* P3 = T3 + kH3 * kLDX;
  float* T2 = P3 + kH3 * kLDX;
  float* P2 = T2 + kH2 * kLDX;
  float* Bs = P2 + kH2 * kLDX;  // [kNKC][160]
  const float inv_al = 1.f / P.celu_alpha;
  const int ty = threadIdx.x >> 5;
  const int ntiles = ws.seg[S] / kTM;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int row0 = tile * kTM;
    int sp = pos4_species(ws.pos4[row0]);
    if (!NNP_IN(sp, P.S, ws.flags)) sp = 0;
    int valid[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) valid[i] = ws.row_atom[row0 + ty * 8 + i] >= 0;
    {  // layer 3: th3 = w4, ph3 = 0
      float th[8][kH3 / 32], ph[8][kH3 / 32];
      const int tx = threadIdx.x & 31;
#pragma unroll
      for (int j = 0; j < kH3 / 32; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          th[i][j] = Wt.W[sp][3][tx + 32 * j];
          ph[i][j] = 0.f;
        }
      fm_store_rev<kH3>(th, ph, z, dz, t, p, T3, P3, row0, fm_off(2), valid, inv_al);
    }
    {  // layer 2: th2 = t3 W3^T, ph2 = p3 W3^T
      f2 a[4][kH2 / 32], ad[4][kH2 / 32];
      net_zero<kH2>(a);
      net_zero<kH2>(ad);
      fm_gemm2<kH2, false>(a, ad, T3, P3, nullptr, nullptr, 0, kH3, Wt.WT[sp][2], Bs, nullptr, nullptr);
      float th[8][kH2 / 32], ph[8][kH2 / 32];
      fm_rows<kH2 / 32>(a, th);
      fm_rows<kH2 / 32>(ad, ph);
      fm_store_rev<kH2>(th, ph, z, dz, t, p, T2, P2, row0, fm_off(1), valid, inv_al);
    }
    {  // layer 1: th1 = t2 W2^T, ph1 = p2 W2^T
      f2 a[4][kH1 / 32], ad[4][kH1 / 32];
      net_zero<kH1>(a);
      net_zero<kH1>(ad);
      fm_gemm2<kH1, false>(a, ad, T2, P2, nullptr, nullptr, 0, kH2, Wt.WT[sp][1], Bs, nullptr, nullptr);
      float th[8][kH1 / 32], ph[8][kH1 / 32];
      fm_rows<kH1 / 32>(a, th);
      fm_rows<kH1 / 32>(ad, ph);
      fm_store_rev<kH1>(th, ph, z, dz, t, p, nullptr, nullptr, row0, fm_off(0), valid, inv_al);
    }
    __syncthreads();
  }
}

// Weight-gradient reduction over the rows of one species.  Job = a 64 x 64
// tile (i0, o0) of layer l's (fan_in x fan_out) gradient, for rows [r0, r1);
// l = 4 means w4 (tile of 64 x 1).  The job's rows go through shared memory
// 32 at a time (the inputs h, dh and the adjoints t, p of the tile); thread
// (ti, to) keeps a 4 x 4 block of the tile (inputs 4 ti.., outputs 4 to..),
// so each row costs it four 16-byte shared loads for 32 FMAs (16 f32x2), and
// each staged value serves 64 products.  FP32 partials over at most 256 rows
// (a job's rows), then one FP64 atomic add per entry into the packed gradient
// (zeroed before).
constexpr int kWgT = 64;       // tile edge (inputs and outputs)
constexpr int kWgRows = 32;    // rows staged at a time
constexpr int kWgLd = kWgT + 4;  // floats per staged row (16-byte aligned 4-column reads)
constexpr int kWgFlush = 8;      // chunks summed in FP32 before each FP64 flush
__global__ void __launch_bounds__(256, 3) k_fm_wgrad(DescParams P, const FmJob* __restrict__ jobs, int njobs,
                                                  const float* __restrict__ G, const float* __restrict__ dG,
                                                  const float* __restrict__ z, const float* __restrict__ dz,
                                                  const float* __restrict__ t, const float* __restrict__ p,
                                                  double* grad) {
  __shared__ __align__(16) float Hc[kWgRows][kWgLd], DHc[kWgRows][kWgLd], Tc[kWgRows][kWgLd], Pc[kWgRows][kWgLd];
  const int D = P.D;
  const float al = P.celu_alpha, inv_al = 1.f / P.celu_alpha;
  const int tid = threadIdx.x;
  const int ti = tid >> 4, to = tid & 15;
  for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
    const FmJob jbv = jobs[jb];
    const int l = jbv.l;
    const int fin = l == 1 ? D : (l == 2 ? kH1 : (l == 3 ? kH2 : kH3));
    const int fout = l == 1 ? kH1 : (l == 2 ? kH2 : (l == 3 ? kH3 : 1));
    f2 a[4][2], b[2];  // a[x][y/2]: outputs (4ti + x, 4to + y), y pairs; b: bias sums
#pragma unroll
    for (int x = 0; x < 4; ++x) a[x][0] = a[x][1] = f2_make(0.f, 0.f);
    b[0] = b[1] = f2_make(0.f, 0.f);
    int chunks = 0;
    const double sc = (double)jbv.scale;
    for (int c0 = jbv.r0; c0 < jbv.r1; c0 += kWgRows) {
      const int nr = min(kWgRows, jbv.r1 - c0);
      __syncthreads();
      for (int e = tid; e < kWgRows * kWgT; e += 256) {
        const int rr = e / kWgT, cc = e % kWgT;
        const int r = c0 + rr, i = jbv.i0 + cc, o = jbv.o0 + cc;
        float hv = 0.f, dhv = 0.f, tv = 0.f, pv = 0.f;
        if (rr < nr) {
          if (i < fin) {
            if (l == 1) {
              hv = G[(size_t)r * D + i];
              dhv = dG[(size_t)r * D + i];
            } else {
              const int off = fm_off(l - 2);
              const float zz = z[(size_t)r * kFmW + off + i];
              hv = celu_f(zz, al, inv_al);
              dhv = dcelu_from_h(hv, inv_al) * dz[(size_t)r * kFmW + off + i];
            }
          }
          if (l < 4 && o < fout) {
            tv = t[(size_t)r * kFmW + fm_off(l - 1) + o];
            pv = p[(size_t)r * kFmW + fm_off(l - 1) + o];
          } else if (l == 4 && cc == 0) {
            tv = 1.f;  // phi = dh_3 . w4: adjoint of w4 is dh_3
          }
        }
        Hc[rr][cc] = hv;
        DHc[rr][cc] = dhv;
        Tc[rr][cc] = tv;
        Pc[rr][cc] = pv;
      }
      __syncthreads();
      for (int rr = 0; rr < nr; ++rr) {
        const float4 h4 = *reinterpret_cast<const float4*>(&Hc[rr][4 * ti]);
        const float4 d4 = *reinterpret_cast<const float4*>(&DHc[rr][4 * ti]);
        const float4 t4 = *reinterpret_cast<const float4*>(&Tc[rr][4 * to]);
        const float4 p4 = *reinterpret_cast<const float4*>(&Pc[rr][4 * to]);
        const float hv[4] = {h4.x, h4.y, h4.z, h4.w}, dv[4] = {d4.x, d4.y, d4.z, d4.w};
        const f2 tp[2] = {f2_make(t4.x, t4.y), f2_make(t4.z, t4.w)};
        const f2 pp[2] = {f2_make(p4.x, p4.y), f2_make(p4.z, p4.w)};
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const f2 hh = f2_make(hv[x], hv[x]), dd = f2_make(dv[x], dv[x]);
#pragma unroll
          for (int y = 0; y < 2; ++y) a[x][y] = f2_fma(dd, tp[y], f2_fma(hh, pp[y], a[x][y]));
        }
        b[0] = f2_add(b[0], pp[0]);
        b[1] = f2_add(b[1], pp[1]);
      }
      // at most 256 rows in FP32, then one FP64 add per entry into the gradient
      if (++chunks == kWgFlush || c0 + kWgRows >= jbv.r1) {
        chunks = 0;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int i = jbv.i0 + 4 * ti + x;
#pragma unroll
          for (int y = 0; y < 2; ++y) {
            const float2 v = f2_split(a[x][y]);
            const int o = jbv.o0 + 4 * to + 2 * y;
            if (i < fin && o < fout) atomicAdd(&grad[jbv.w_off + (size_t)i * fout + o], -sc * (double)v.x);
            if (i < fin && o + 1 < fout) atomicAdd(&grad[jbv.w_off + (size_t)i * fout + o + 1], -sc * (double)v.y);
            a[x][y] = f2_make(0.f, 0.f);
          }
        }
        if (ti == 0 && jbv.i0 == 0 && l < 4)
#pragma unroll
          for (int y = 0; y < 2; ++y) {
            const float2 v = f2_split(b[y]);
            const int o = jbv.o0 + 4 * to + 2 * y;
            if (o < fout) atomicAdd(&grad[jbv.b_off + o], -sc * (double)v.x);
            if (o + 1 < fout) atomicAdd(&grad[jbv.b_off + o + 1], -sc * (double)v.y);
          }
        b[0] = b[1] = f2_make(0.f, 0.f);
      }
    }
  }
}

size_t fm_fwd_smem(int /*D*/) {
  return sizeof(float) * ((size_t)(2 * kH1 + 2 * kH2) * kLDX + (size_t)kNKC * kH1 + (size_t)2 * kNKC * kLDX);
}
size_t fm_rev_smem() {
  return sizeof(float) * ((size_t)(2 * kH3 + 2 * kH2) * kLDX + (size_t)kNKC * kH1);
}

void launch_fm(int grid, cudaStream_t st, const DescParams& P, const Workspace& ws, const MlpF32Weights& W,
               const float* dG, float* z, float* dz, float* t, float* p) {
  const size_t sf = fm_fwd_smem(P.D), sr = fm_rev_smem();
#define FM(s) k_fm_fwd<s><<<grid, 256, sf, st>>>(P, ws, W, dG, z, dz); k_fm_rev<s><<<grid, 256, sr, st>>>(P, ws, W, z, dz, t, p)
  switch (P.S) { NNP_SPECIES_CASES(FM) }
#undef FM
}

void launch_fm_wgrad(int grid, cudaStream_t st, const DescParams& P, const FmJob* jobs, int njobs,
                     const float* G, const float* dG, const float* z, const float* dz, const float* t,
                     const float* p, double* grad) {
  k_fm_wgrad<<<grid, 256, 0, st>>>(P, jobs, njobs, G, dG, z, dz, t, p, grad);
}

size_t mlp_f32_smem(int) {
  return sizeof(float) * ((size_t)(kH1 + kH2 + kH3) * kLDX + (size_t)kNKC * kNBsN);
}

void launch_mlp_f32(int grid, cudaStream_t st, const EvalIO* io, const DescParams& P,
                    const Workspace& ws, const MlpF32Weights& W, int acc) {
  const size_t sm = mlp_f32_smem(P.D);
  // grid: one CTA per SM (or per tile, if fewer); two are resident per SM
  grid *= 2;
#define MLP(s) k_mlp_f32<s><<<grid, 256, sm, st>>>(io, P, ws, W, acc)
  switch (P.S) { NNP_SPECIES_CASES(MLP) }
#undef MLP
}

cudaError_t mlp_f32_set_smem_limits() {
  cudaError_t e;
#define MSM(s) e = cudaFuncSetAttribute(k_mlp_f32<s>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    (int)mlp_f32_smem(desc_len(s))); if (e) return e
  MSM(1); MSM(2); MSM(3); MSM(4); MSM(5); MSM(6); MSM(7); MSM(8);
#undef MSM
  const void* fwd[kMaxS] = {(const void*)k_fm_fwd<1>, (const void*)k_fm_fwd<2>, (const void*)k_fm_fwd<3>,
                            (const void*)k_fm_fwd<4>, (const void*)k_fm_fwd<5>, (const void*)k_fm_fwd<6>,
                            (const void*)k_fm_fwd<7>, (const void*)k_fm_fwd<8>};
  const void* rev[kMaxS] = {(const void*)k_fm_rev<1>, (const void*)k_fm_rev<2>, (const void*)k_fm_rev<3>,
                            (const void*)k_fm_rev<4>, (const void*)k_fm_rev<5>, (const void*)k_fm_rev<6>,
                            (const void*)k_fm_rev<7>, (const void*)k_fm_rev<8>};
  for (int q = 0; q < kMaxS; ++q) {
    e = cudaFuncSetAttribute(fwd[q], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fm_fwd_smem(desc_len(q + 1))); if (e) return e;
    e = cudaFuncSetAttribute(rev[q], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fm_rev_smem()); if (e) return e;
  }
  return e;
}

}  // namespace nnp
