// k_mlp_f32.cu -- per-element network, FP32 form (SIMT FFMA), fused:
// forward D -> 160 -> 128 -> 96 -> 1 with CELU, the atom energies E_i and
// their sum per system (FP64), and the backward pass to dE_i/dG_i (the first
// factor of the force chain rule, Eq. 2).
//
//   h_l = CELU(h_{l-1} W_l + b_l),  E_i = h_3 w_4 + b_4
//   g_3 = w_4 * CELU'(z_3),  g_{l-1} = (g_l W_l^T) * CELU'(z_{l-1}),
//   dE/dG = g_1 W_1^T,   CELU'(z) = 1 (z > 0), h/alpha + 1 (z <= 0)
//
// One CTA of 256 threads per 64-row tile (one species per tile).  Thread
// (warp ty, lane tx) owns rows 8ty..8ty+7 and columns tx + 32j.  The tile's
// activations stay in shared memory, transposed (feature-major, padded
// leading dimension) so that a thread's 8 rows are two float4 loads;
// weights stream through a shared chunk buffer.
#include "nnp_internal.cuh"

namespace nnp {

constexpr int kTM = 64;          // rows per tile
constexpr int kLDX = kTM + 4;    // padded leading dim of transposed activations
constexpr int kKC = 32;          // streamed k-chunk

// acc[8][NJ] += A(64 x K) * B(K x N).  A is either transposed in shared
// memory (AT[k][kLDX]) or, if Ag != nullptr, rows of global memory (lda).
template <int N>
__device__ __forceinline__ void gemm_tile(float (&acc)[8][(N + 31) / 32], const float* AT,
                                          const float* __restrict__ Ag, int lda, int K,
                                          const float* __restrict__ Bg, float* Bs, float* As) {
  constexpr int NJ = (N + 31) / 32;
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  for (int k0 = 0; k0 < K; k0 += kKC) {
    const int kc = min(kKC, K - k0);
    __syncthreads();
    for (int i = tid; i < kc * N; i += 256) Bs[i] = Bg[(size_t)k0 * N + i];
    if (Ag) {
      for (int i = tid; i < kTM * kc; i += 256) {
        const int r = i / kc, kk = i - r * kc;
        As[kk * kLDX + r] = Ag[(size_t)r * lda + k0 + kk];
      }
    }
    __syncthreads();
    const float* Ab = Ag ? As : AT + (size_t)k0 * kLDX;
#pragma unroll 4
    for (int kk = 0; kk < kc; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(Ab + kk * kLDX + ty * 8);
      const float4 a1 = *reinterpret_cast<const float4*>(Ab + kk * kLDX + ty * 8 + 4);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float b[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int col = tx + 32 * j;
        b[j] = (N % 32 == 0 || col < N) ? Bs[kk * N + col] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
}

template <int N>
__device__ __forceinline__ void zero_acc(float (&acc)[8][(N + 31) / 32]) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < (N + 31) / 32; ++j) acc[i][j] = 0.f;
}

__device__ __forceinline__ float celu_f(float z, float al, float inv_al) {
  return z > 0.f ? z : al * (expf(z * inv_al) - 1.f);
}
// CELU'(z) from h = CELU(z): 1 for h > 0, h/alpha + 1 otherwise
__device__ __forceinline__ float dcelu_from_h(float h, float inv_al) {
  return h > 0.f ? 1.f : fmaf(h, inv_al, 1.f);
}

// Forward layer epilogue: H^T[col][row] = CELU(acc + b)
template <int N>
__device__ __forceinline__ void store_celu(const float (&acc)[8][(N + 31) / 32], const float* bias,
                                           float* HT, float al, float inv_al) {
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < (N + 31) / 32; ++j) {
    const int col = tx + 32 * j;
    if (N % 32 != 0 && col >= N) continue;
    const float bb = bias[col];
    float h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = celu_f(acc[i][j] + bb, al, inv_al);
    *reinterpret_cast<float4*>(HT + col * kLDX + ty * 8) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(HT + col * kLDX + ty * 8 + 4) = make_float4(h[4], h[5], h[6], h[7]);
  }
}

// Backward epilogue: HT[col][row] <- acc * CELU'(h) where h = HT[col][row]
template <int N>
__device__ __forceinline__ void store_bwd(const float (&acc)[8][(N + 31) / 32], float* HT,
                                          float inv_al) {
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < (N + 31) / 32; ++j) {
    const int col = tx + 32 * j;
    float4* p0 = reinterpret_cast<float4*>(HT + col * kLDX + ty * 8);
    float4* p1 = p0 + 1;
    const float4 h0 = *p0, h1 = *p1;
    const float h[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
    float g[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) g[i] = acc[i][j] * dcelu_from_h(h[i], inv_al);
    *p0 = make_float4(g[0], g[1], g[2], g[3]);
    *p1 = make_float4(g[4], g[5], g[6], g[7]);
  }
}

template <int S>
__global__ void __launch_bounds__(256, 1) k_mlp_f32(const EvalIO* __restrict__ io,
                                                    DescParams P, Workspace ws, MlpF32Weights Wt) {
  constexpr int D = kNRad * S + kNAng * S * (S + 1) / 2;
  extern __shared__ float smf[];
  float* H1T = smf;                       // [160][kLDX]
  float* H2T = H1T + kH1 * kLDX;          // [128][kLDX]
  float* H3T = H2T + kH2 * kLDX;          // [96][kLDX]
  float* Bs = H3T + kH3 * kLDX;           // [kKC][max N = max(160, D)]
  constexpr int kBsN = (D > kH1 ? D : kH1);
  float* As = Bs + kKC * kBsN;            // [kKC][kLDX]
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
  const float al = P.celu_alpha, inv_al = 1.f / P.celu_alpha;
  const int rows = ws.seg[S];
  const int ntiles = rows / kTM;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int row0 = tile * kTM;
    const int sp = pos4_species(ws.pos4[row0]);
    // ---- forward
    float acc1[8][kH1 / 32];
    zero_acc<kH1>(acc1);
    gemm_tile<kH1>(acc1, nullptr, ws.G + (size_t)row0 * D, D, D, Wt.W[sp][0], Bs, As);
    store_celu<kH1>(acc1, Wt.b[sp][0], H1T, al, inv_al);
    float acc2[8][kH2 / 32];
    zero_acc<kH2>(acc2);
    gemm_tile<kH2>(acc2, H1T, nullptr, 0, kH1, Wt.W[sp][1], Bs, As);
    store_celu<kH2>(acc2, Wt.b[sp][1], H2T, al, inv_al);
    float acc3[8][kH3 / 32];
    zero_acc<kH3>(acc3);
    gemm_tile<kH3>(acc3, H2T, nullptr, 0, kH2, Wt.W[sp][2], Bs, As);
    // layer 3 epilogue: energy and g3 = w4 * CELU'(z3), stored in H3T
    {
      const float* w4 = Wt.W[sp][3];
      const float* b3 = Wt.b[sp][2];
      float e[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) e[i] = 0.f;
#pragma unroll
      for (int j = 0; j < kH3 / 32; ++j) {
        const int col = tx + 32 * j;
        const float ww = w4[col], bb = b3[col];
        float g[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float z = acc3[i][j] + bb;
          const float h = celu_f(z, al, inv_al);
          e[i] = fmaf(h, ww, e[i]);
          g[i] = ww * (z > 0.f ? 1.f : expf(z * inv_al));
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
      if (tx < 8) ws.Ei[row] = valid ? ev : 0.f;
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
    // ---- backward
    float accb2[8][kH2 / 32];
    zero_acc<kH2>(accb2);
    gemm_tile<kH2>(accb2, H3T, nullptr, 0, kH3, Wt.WT[sp][2], Bs, As);
    store_bwd<kH2>(accb2, H2T, inv_al);
    float accb1[8][kH1 / 32];
    zero_acc<kH1>(accb1);
    gemm_tile<kH1>(accb1, H2T, nullptr, 0, kH2, Wt.WT[sp][1], Bs, As);
    store_bwd<kH1>(accb1, H1T, inv_al);
    float accg[8][(D + 31) / 32];
    zero_acc<D>(accg);
    gemm_tile<D>(accg, H1T, nullptr, 0, kH1, Wt.WT[sp][0], Bs, As);
#pragma unroll
    for (int j = 0; j < (D + 31) / 32; ++j) {
      const int col = tx + 32 * j;
      if (D % 32 != 0 && col >= D) continue;
#pragma unroll
      for (int i = 0; i < 8; ++i) ws.dEdG[(size_t)(row0 + ty * 8 + i) * D + col] = accg[i][j];
    }
    __syncthreads();
  }
}

size_t mlp_f32_smem(int D) {
  const int bsn = D > kH1 ? D : kH1;
  return sizeof(float) * ((size_t)(kH1 + kH2 + kH3) * kLDX + (size_t)kKC * bsn + (size_t)kKC * kLDX);
}

void launch_mlp_f32(int grid, cudaStream_t st, const EvalIO* io, const DescParams& P,
                    const Workspace& ws, const MlpF32Weights& W) {
  const size_t sm = mlp_f32_smem(P.D);
  switch (P.S) {
    case 1: k_mlp_f32<1><<<grid, 256, sm, st>>>(io, P, ws, W); break;
    case 2: k_mlp_f32<2><<<grid, 256, sm, st>>>(io, P, ws, W); break;
    case 3: k_mlp_f32<3><<<grid, 256, sm, st>>>(io, P, ws, W); break;
    default: k_mlp_f32<4><<<grid, 256, sm, st>>>(io, P, ws, W); break;
  }
}

cudaError_t mlp_f32_set_smem_limits() {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_mlp_f32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_f32_smem(48)); if (e) return e;
  e = cudaFuncSetAttribute(k_mlp_f32<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_f32_smem(128)); if (e) return e;
  e = cudaFuncSetAttribute(k_mlp_f32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_f32_smem(240)); if (e) return e;
  e = cudaFuncSetAttribute(k_mlp_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_f32_smem(384));
  return e;
}

}  // namespace nnp
