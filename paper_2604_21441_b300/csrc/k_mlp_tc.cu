// k_mlp_tc.cu -- per-element network on the 5th-generation tensor cores
// (tcgen05.mma, BF16 or FP8 operands, FP32 accumulators in tensor memory), fused:
// forward D -> 160 -> 128 -> 96 -> 1 with CELU, atom energies and their FP64
// sum per system, and the backward pass to dE_i/dG_i (chain rule of Eq. 2):
//
//   z_l = h_{l-1} W_l + b_l, h_l = CELU(z_l), E_i = h_3 w_4 + b_4
//   g_3 = w_4 * CELU'(z_3), g_{l-1} = (g_l W_l^T) * CELU'(z_{l-1}), dE/dG = g_1 W_1^T
//
// One CTA (16 warps) per SM, persistent over 128-row tiles (one species per
// tile).  Row r of a tile is TMEM lane r; warps w, w+4, w+8 and w+12 share the
// lanes of quarter w and split each epilogue's 16-column chunks.  Thread 0 issues the
// bulk (TMA) copies and the MMAs; all threads run the epilogues, reading
// biases from shared memory and keeping two TMEM loads in flight.
// Shared memory holds three activation buffers and two weight buffers, every
// operand in the K-major 128-byte-swizzled layout (slabs of 64 columns x 128
// rows, 16-byte chunk j of row r stored at chunk j ^ (r & 7)).  The descriptor
// tile arrives in that layout from the descriptor kernel; the six weight
// matrices per species are pre-swizzled on the host.  The next weight matrix
// streams in while the current layer runs.
//
// TMEM columns (512 allocated): z1 [0,160)  z2 [160,288)  z3 [288,384)
// g2' [384,512)  g1' [160,320)  dE/dG [384, 384 + D).  The forward epilogues
// overwrite z1 and z2 with CELU'(z1), CELU'(z2) in FP32, which the backward
// epilogues multiply in; the backward does not lose precision to the BF16
// activations and does not evaluate the exponential again.  Because dE/dG
// sits above column 384, the next tile's layer-1 MMA (into [0,160)) is issued
// as soon as this tile's last MMA is done and runs under the dE/dG epilogue.
//
// FP8 form: the three forward GEMMs take E4M3 operands (kind::f8f6f4, twice
// the BF16 rate) with static scales: activations x_q = x / s_x with one s_x
// per layer, species and ensemble member from a calibration pass of the FP32
// form over the first input; weights W_q[., n] = W[., n] / s_W[n] with one
// scale per output column and member, s_W[n] = max_k |W[k, n]| / 448.  The accumulator of column n is
// rescaled by s_x s_W[n] in the epilogue, before the bias.  The backward
// GEMMs stay BF16; CELU' comes from the FP8 forward's z.
//
// Every wait on an mbarrier is bounded; on timeout the kernel raises the
// timeout flag, stops issuing work, waits (bounded) for its own copies and
// MMAs, frees its tensor memory and returns.
#include <cmath>
#include <cstring>
#include <vector>

#include "nnp_host.h"

namespace nnp {

namespace {

constexpr int kTM = 128;                 // rows per tile (MMA M)
constexpr int kTcThreads = 512;          // 16 warps: 4 per TMEM lane quarter
constexpr int kG = kTcThreads / 128;     // column groups of the epilogues
constexpr int kSlab = kTM * 128;         // bytes of one 64-column slab
constexpr uint32_t kTmemCols = 512;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on any wait

__host__ __device__ constexpr int slabs_of(int K) { return (K + 63) / 64; }
__host__ __device__ constexpr int mat_bytes(int N, int K) { return slabs_of(K) * N * 128; }
// FP8 operands: 128 one-byte K columns per slab
__host__ __device__ constexpr int slabs8_of(int K) { return (K + 127) / 128; }
__host__ __device__ constexpr int mat8_bytes(int N, int K) { return slabs8_of(K) * N * 128; }

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of the given parity; false after limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  for (int i = 0; i < 64; ++i)  // short waits without reading the timer
    if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) { return mbar_wait_for(bar, parity, kWaitNs); }
// The same bound for threads that only wait (epilogue threads while thread 0
// streams operands and issues MMAs): they back off with nanosleep between
// tries, so that their polling does not take issue slots from the thread
// that does the work.
__device__ __forceinline__ bool mbar_wait_idle(uint64_t* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  unsigned ns = 32;
  while (!mbar_try(bar, parity)) {
    if (global_ns() - t0 > kWaitNs) return false;
    __nanosleep(ns);
    ns = ns < 256 ? 2 * ns : 256;
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// K-major operand, 128-byte swizzle: start address, leading byte offset
// (unused for this layout, 16 B), stride byte offset 1024 B between 8-row
// groups, fixed version bits 0b001 at [46,49), swizzle mode 2 at [61,64).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// kind::f8f6f4 instruction descriptor: FP32 accumulate, E4M3 A and B (format
// code 0 in both fields), both K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[128 x N] = A[128 x K] B[N x K]^T.  One MMA covers 32 bytes of K (16 BF16
// or 32 E4M3 values), so both types advance 32 bytes per MMA inside a
// 128-byte swizzle row and one slab per four MMAs.
// acc0 = 1: the first MMA adds to D as well (a later K chunk of one product).
template <bool F8>
__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, const uint8_t* A, const uint8_t* B, int N, int K,
                                           uint32_t acc0 = 0u) {
  const uint32_t idesc = F8 ? idesc_e4m3(kTM, N) : idesc_bf16(kTM, N);
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
  const int nk = K / (F8 ? 32 : 16);
  for (int k = 0; k < nk; ++k) {
    const uint32_t a = a0 + (uint32_t)(k >> 2) * kSlab + (uint32_t)(k & 3) * 32;
    const uint32_t b = b0 + (uint32_t)(k >> 2) * (uint32_t)(N * 128) + (uint32_t)(k & 3) * 32;
    if (F8) mma_e4m3(d_tmem, sw128_desc(a), sw128_desc(b), idesc, (k > 0 || acc0) ? 1u : 0u);
    else mma_bf16(d_tmem, sw128_desc(a), sw128_desc(b), idesc, (k > 0 || acc0) ? 1u : 0u);
  }
}

// CELU and its derivative; k = log2(e) / alpha, so exp(z / alpha) = exp2(k z).
// 2^x on the MUFU unit; results below the normal range flush to zero, which
// moves CELU(z) = alpha (e^(z/alpha) - 1) by less than alpha 2^-126.
__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Store 16 values of row r, columns [c0, c0+16), as BF16 into a swizzled buffer.
__device__ __forceinline__ void store_row16(uint8_t* buf, int r, int c0, const float (&v)[16]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int ch = (c0 >> 3) + h;  // 16-byte chunk index along K
    uint4 q;
    __nv_bfloat162 p0 = __floats2bfloat162_rn(v[8 * h + 0], v[8 * h + 1]);
    __nv_bfloat162 p1 = __floats2bfloat162_rn(v[8 * h + 2], v[8 * h + 3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(v[8 * h + 4], v[8 * h + 5]);
    __nv_bfloat162 p3 = __floats2bfloat162_rn(v[8 * h + 6], v[8 * h + 7]);
    q.x = *reinterpret_cast<uint32_t*>(&p0);
    q.y = *reinterpret_cast<uint32_t*>(&p1);
    q.z = *reinterpret_cast<uint32_t*>(&p2);
    q.w = *reinterpret_cast<uint32_t*>(&p3);
    uint8_t* dst = buf + (ch >> 3) * kSlab + r * 128 + (((ch & 7) ^ (r & 7)) << 4);
    *reinterpret_cast<uint4*>(dst) = q;
  }
}

// Store 16 values of row r, columns [c0, c0+16), times q as E4M3 (one 16-byte chunk).
__device__ __forceinline__ void store_row16_e4m3(uint8_t* buf, int r, int c0, const float (&v)[16], float q) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i] * q, v[4 * i + 1] * q), __NV_SATFINITE,
                                                 __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[4 * i + 2] * q, v[4 * i + 3] * q),
                                                 __NV_SATFINITE, __NV_E4M3);
    w[i] = lo | (hi << 16);
  }
  const int ch = c0 >> 4;  // 16-byte chunk index along K
  uint8_t* dst = buf + (ch >> 3) * kSlab + r * 128 + (((ch & 7) ^ (r & 7)) << 4);
  *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

}  // namespace

// Pre-swizzled weights per species: forward W1^T (160 x D), W2^T
// (128 x 160), W3^T (96 x 128); backward W3 (128 x 96), W2 (160 x 128),
// W1 (D x 160); each [N rows x K cols], K-major.
struct MlpTcWeights {
  const uint8_t* m[kMaxS][6];
  const float* wsc[kMaxS];  // FP8: per-output-column scales s_W[n] of W1, W2, W3 (160 + 128 + 96)
};

// Per-system energy sums of one warp's 32 rows: rows of a system are
// contiguous, so each run is summed by shuffles and added once in FP64.
__device__ __forceinline__ void tile_energy_sums(float e, bool valid, int sys, int lane, double* energies) {
  unsigned todo = __ballot_sync(0xffffffffu, valid);
  while (todo) {
    const int leader = __ffs(todo) - 1;
    const int ls = __shfl_sync(0xffffffffu, sys, leader);
    const bool mine = valid && sys == ls;
    float x = mine ? e : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == leader) atomicAdd(&energies[ls], (double)x);
    todo &= ~__ballot_sync(0xffffffffu, mine);
  }
}

// *o += (x, y, z, w): one vector reduction in global memory (L2)
__device__ __forceinline__ void red_add_v4(float4* o, float x, float y, float z, float w) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(o), "f"(x), "f"(y), "f"(z), "f"(w)
               : "memory");
}

// Issue the TMEM load of 16 columns (no wait).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]);
__device__ __forceinline__ void tmem_wait_ld();

// Epilogue of an accumulator block of ncols (<= 128, a multiple of 16)
// columns: the warp's 32 rows (TMEM lanes) x columns [32 h, 32 h + 32) go
// through a warp-private staging area of 32 x 8 float4 (4 KB; float4 k of row
// r at r * 8 + (k ^ (r & 7)), so that neither the row-per-lane writes nor the
// row-by-row reads conflict on banks) and leave as whole 128-byte lines:
// eight lanes per row, four rows per instruction.  out points at column 0 of
// the warp's first row, ld is the row stride; acc = 1 adds with FP32
// vector reductions, 0 stores.
__device__ __forceinline__ void store_block_staged(uint32_t tcol, int h, int lane, float* out, int ld,
                                                   int ncols, float4* stage, int acc) {
  const int c0 = 32 * h;
  if (c0 >= ncols) return;  // warp-uniform
  const bool two = c0 + 16 < ncols;
  uint32_t a[16], b[16];
  tmem_ld16_nowait(tcol + c0, a);
  if (two) tmem_ld16_nowait(tcol + c0 + 16, b);
  tmem_wait_ld();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    stage[lane * 8 + (k ^ (lane & 7))] = make_float4(__uint_as_float(a[4 * k]), __uint_as_float(a[4 * k + 1]),
                                                     __uint_as_float(a[4 * k + 2]), __uint_as_float(a[4 * k + 3]));
    if (two)
      stage[lane * 8 + ((k + 4) ^ (lane & 7))] =
          make_float4(__uint_as_float(b[4 * k]), __uint_as_float(b[4 * k + 1]), __uint_as_float(b[4 * k + 2]),
                      __uint_as_float(b[4 * k + 3]));
  }
  __syncwarp();
  const int kk = lane & 7, nk = two ? 8 : 4;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int row = 4 * j + (lane >> 3);
    if (kk < nk) {
      const float4 v = stage[row * 8 + (kk ^ (row & 7))];
      float4* o = reinterpret_cast<float4*>(out + (size_t)row * ld + c0 + 4 * kk);
      if (acc) red_add_v4(o, v.x, v.y, v.z, v.w);
      else *o = v;
    }
  }
  __syncwarp();  // the staging area is read before the warp writes it again
}
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Store 16 columns of the warp's 32 lanes to TMEM (completion: tmem_wait_st).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Epilogue skeleton: the warp's column group h handles 16-column chunks
// h, h + kG, ...; two chunks are loaded from TMEM per wait.
// f(chunk_col0, values[16]).
template <int N, class F>
__device__ __forceinline__ void for_chunks(uint32_t tcol, int h, F f) {
  constexpr int NCH = N / 16;
  for (int c = h; c < NCH; c += 2 * kG) {
    uint32_t a[16], b[16];
    const bool two = c + kG < NCH;
    tmem_ld16_nowait(tcol + c * 16, a);
    if (two) tmem_ld16_nowait(tcol + (c + kG) * 16, b);
    tmem_wait_ld();
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(a[j]);
    f(c * 16, v);
    if (two) {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(b[j]);
      f((c + kG) * 16, v);
    }
  }
}

// Same, with a second TMEM operand (the pre-activation) per chunk.
template <int N, class F>
__device__ __forceinline__ void for_chunks2(uint32_t tcol, uint32_t tcol2, int h, F f) {
  constexpr int NCH = N / 16;
  for (int c = h; c < NCH; c += kG) {
    uint32_t a[16], b[16];
    tmem_ld16_nowait(tcol + c * 16, a);
    tmem_ld16_nowait(tcol2 + c * 16, b);
    tmem_wait_ld();
    float g[16], z[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      g[j] = __uint_as_float(a[j]);
      z[j] = __uint_as_float(b[j]);
    }
    f(c * 16, g, z);
  }
}

// Work items are (tile, member) pairs for members m0 .. m0 + nm - 1 of the
// weight sets Wts / Wfs (device arrays), member-minor: the members of one
// tile are consecutive items, so they run at the same time on neighbouring
// CTAs, which read the tile's descriptor rows from DRAM once between them
// and whose dE/dG reductions meet in L2.  accm =
// 1: E_i and dE/dG are added with reductions into buffers the caller zeroed
// (members running side by side); 0: written.
template <int D, bool F8>
__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_tc(const EvalIO* __restrict__ io, DescParams P,
                                                  Workspace ws, const MlpTcWeights* __restrict__ Wts,
                                                  const MlpF32Weights* __restrict__ Wfs, int m0, int nm,
                                                  int accm) {
  constexpr int kBufA = slabs_of(D > kH2 ? D : kH2) * kSlab;  // G, later g2
  constexpr int kBufB = slabs_of(kH1) * kSlab;                // h1, later g1
  constexpr int kBufC = slabs_of(kH2) * kSlab;                // h2, later g3
  constexpr int kWBuf = 48 * 1024;
  static_assert(mat_bytes(kH1, D) <= kWBuf && mat_bytes(D, kH1) <= kWBuf, "weight buffer");
  static_assert(D % (F8 ? 32 : 16) == 0, "D must be a multiple of one MMA's K");
  constexpr int NW[6] = {kH1, kH2, kH3, kH2, kH1, D};  // N of the six GEMMs
  constexpr int KW[6] = {D, kH1, kH2, kH3, kH2, kH1};  // K of the six GEMMs
  constexpr int kNB = kH1 + kH2 + kH3 + kH3 + 1;       // b1 b2 b3 w4 b4

  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* bufA = sm;
  uint8_t* bufB = bufA + kBufA;
  uint8_t* bufC = bufB + kBufB;
  uint8_t* wbuf[2] = {bufC + kBufC, bufC + kBufC + kWBuf};
  // [0,1] weights, [2] tile, [3] MMAs, [4] layer-1 MMAs (may be issued one tile ahead)
  uint64_t* bars = reinterpret_cast<uint64_t*>(wbuf[1] + kWBuf);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 5);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  float* sE = reinterpret_cast<float*>(abort_flag + 1);  // [kG][kTM] partial energies
  float* sb = sE + kG * kTM;  // [kNB] biases and w4 of the tile's species
  float* sb1 = sb;
  float* sb2 = sb1 + kH1;
  float* sb3 = sb2 + kH2;
  float* sw4 = sb3 + kH3;
  float* sb4 = sw4 + kH3;
  float* ssc = sb + kNB;     // FP8: [kH1 + kH2 + kH3] per-column dequantisation s_x s_W[n]
  float* ssc1 = ssc;
  float* ssc2 = ssc1 + kH1;
  float* ssc3 = ssc2 + kH2;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, h = warp >> 2;  // TMEM lane quarter; column group
  const int r = quarter * 32 + lane;            // row of the tile (TMEM lane)
  const float al = P.celu_alpha, kexp = 1.4426950408889634f / P.celu_alpha;
  const int rows = ws.seg[P.S];
  const int ntiles = rows / kTM;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    mbar_init(&bars[3], 1);
    mbar_init(&bars[4], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lb = (uint32_t)(quarter * 32) << 16;
  const uint32_t tz1 = tmem + lb + 0, tz2 = tmem + lb + 160, tz3 = tmem + lb + 288,
                 tg2 = tmem + lb + 384, tg1 = tmem + lb + 160, tdg = tmem + lb + 384;
  const uint32_t mz1 = tmem + 0, mz2 = tmem + 160, mz3 = tmem + 288, mg2 = tmem + 384, mg1 = tmem + 160,
                 mdg = tmem + 384;  // MMA destinations (lane 0)

  // barrier parities and outstanding work: bars 0,1 weights, 2 tile (thread 0
  // waits on these); bar 3 MMA completion (every thread waits on it)
  uint32_t ph[4] = {0, 0, 0, 0};
  bool pend[4] = {false, false, false, false};

  const MlpTcWeights* cur_w = Wts + m0;  // the current work item's member
  const MlpF32Weights* cur_f = Wfs + m0;
  auto load_wm = [&](const MlpTcWeights& W, int sp, int which, int b) {
    const int bytes = (F8 && which < 3) ? mat8_bytes(NW[which], KW[which]) : mat_bytes(NW[which], KW[which]);
    mbar_expect_tx(&bars[b], (uint32_t)bytes);
    bulk_g2s(wbuf[b], W.m[sp][which], (uint32_t)bytes, &bars[b]);
    pend[b] = true;
  };
  auto load_w = [&](int sp, int which, int b) { load_wm(*cur_w, sp, which, b); };
  auto load_tile = [&](int t) {
    const uint32_t bytes = (uint32_t)(F8 ? gh8_tile_bytes(D) : gh_tile_bytes(D));
    mbar_expect_tx(&bars[2], bytes);
    bulk_g2s(bufA, reinterpret_cast<const uint8_t*>(ws.Gh) + (size_t)t * bytes, bytes, &bars[2]);
    pend[2] = true;
  };
  auto commit = [&]() {
    mma_commit(&bars[3]);
    pend[3] = true;
  };
  auto wait0 = [&](int i) {  // thread 0: copies into buffer i have landed
    if (!pend[i]) return;
    if (mbar_wait(&bars[i], ph[i])) {
      ph[i] ^= 1u;
      pend[i] = false;
    } else {
      *abort_flag = 1;
      atomicOr(&ws.flags[kFlagTimeout], 1);
    }
  };
  // Phase boundary: the epilogue's shared-memory writes (generic proxy) and
  // TMEM reads are ordered before the next MMA; thread 0 has seen buffers i
  // and j (-1: none) land; one block barrier publishes both.
  auto phase = [&](int i, int j) -> bool {
    tmem_wait_st();
    fence_proxy_async();
    tc_fence_before();
    if (tid == 0) {
      if (i >= 0) wait0(i);
      if (j >= 0) wait0(j);
    }
    __syncthreads();
    return *abort_flag == 0;
  };
  // every thread waits for the MMAs committed to barrier b (3, or 4 for
  // layer 1); a timeout raises the abort flag and the next phase boundary
  // then ends the loop for all threads
  uint32_t ph4 = 0;
  bool pend4 = false, l1_issued = false;  // thread 0: layer-1 MMA of the current tile in flight
  auto commit4 = [&]() {
    mma_commit(&bars[4]);
    pend4 = true;
  };
  auto wait_mma = [&](int b) {
    uint32_t& p = b == 4 ? ph4 : ph[3];
    if (warp == 0) __syncwarp();  // lanes 1-31 do not poll beside thread 0 while it issues
    if (mbar_wait(&bars[b], p)) {
      p ^= 1u;
      if (tid == 0) {
        if (b == 4) pend4 = false;
        else pend[3] = false;
      }
    } else {
      *abort_flag = 1;
      atomicOr(&ws.flags[kFlagTimeout], 1);
    }
    tc_fence_after();
  };

  const int nwork = ntiles * nm;
  int wi = blockIdx.x;
  if (wi < nwork && tid == 0) {
    const int t0 = wi / nm;
    load_tile(t0);
    load_wm(Wts[m0 + wi % nm], pos4_species(ws.pos4[t0 * kTM]), 0, 0);
  }
  for (; wi < nwork; wi += gridDim.x) {
    const int tile = wi / nm;
    cur_w = Wts + m0 + wi % nm;
    cur_f = Wfs + m0 + wi % nm;
    const int row0 = tile * kTM;
    int sp = pos4_species(ws.pos4[row0]);
    if (!NNP_IN(sp, P.S, ws.flags)) sp = 0;
    const int nwi = wi + gridDim.x;
    const bool has_next = nwi < nwork;
    const int next = has_next ? nwi / nm : 0;
    const MlpTcWeights& next_w = Wts[m0 + (has_next ? nwi % nm : 0)];
    const int sp_next = has_next ? pos4_species(ws.pos4[next * kTM]) : 0;
    const int row = row0 + r;
    const int my_atom = ws.row_atom[row];  // consumed by the energy epilogue
    const int my_sys = ws.row_info[row];
    // FP8: z_l[n] = acc_l[n] * s_x s_W[n] + b_l[n]; q_l = 1 / s_{h_l} quantises h_l
    float q1 = 1.f, q2 = 1.f;
    if (F8) {
      const int* qs = ws.q8 + 8 * ((size_t)(m0 + wi % nm) * kMaxS + sp);  // this member's ranges
      if (tid == 0 && qs[0] == 0) atomicOr(&ws.flags[kFlagFp8Uncal], 1);  // the host calibrates and redoes
      const float sx0 = fp8_step(qs[0]), sx1 = fp8_step(qs[1]), sx2 = fp8_step(qs[2]);
      q1 = 1.f / sx1;
      q2 = 1.f / sx2;
      for (int i = tid; i < kH1 + kH2 + kH3; i += blockDim.x)
        ssc[i] = cur_w->wsc[sp][i] * (i < kH1 ? sx0 : (i < kH1 + kH2 ? sx1 : sx2));
    }
    for (int i = tid; i < kNB; i += blockDim.x) {
      float v;
      if (i < kH1) v = cur_f->b[sp][0][i];
      else if (i < kH1 + kH2) v = cur_f->b[sp][1][i - kH1];
      else if (i < kH1 + kH2 + kH3) v = cur_f->b[sp][2][i - kH1 - kH2];
      else if (i < kH1 + kH2 + 2 * kH3) v = cur_f->W[sp][3][i - kH1 - kH2 - kH3];
      else v = cur_f->b[sp][3][0];
      sb[i] = v;
    }
    // ---------------- layer 1: z1 = G W1
    if (!phase(2, 0)) break;                         // G tile, W1^T in wbuf[0] (also publishes sb)
    if (tid == 0) {
      load_w(sp, 1, 1);                              // W2^T -> wbuf[1]
      if (!l1_issued) {
        tc_fence_after();
        issue_gemm<F8>(mz1, bufA, wbuf[0], kH1, D);
        commit4();
      }
      l1_issued = false;
    }
    wait_mma(4);
    for_chunks<kH1>(tz1, h, [&](int c0, float (&v)[16]) {
      float d[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float z = fmaf(v[j], F8 ? ssc1[c0 + j] : 1.f, sb1[c0 + j]);
        const float ez = ex2f(z * kexp);
        v[j] = z > 0.f ? z : al * (ez - 1.f);
        d[j] = z > 0.f ? 1.f : ez;
      }
      tmem_st16(tz1 + c0, d);  // CELU'(z1) for the backward
      if (F8) store_row16_e4m3(bufB, r, c0, v, q1);
      else store_row16(bufB, r, c0, v);
    });
    // ---------------- layer 2: z2 = h1 W2
    if (!phase(1, -1)) break;
    if (tid == 0) {
      load_w(sp, 2, 0);                              // W3^T -> wbuf[0]
      tc_fence_after();
      issue_gemm<F8>(mz2, bufB, wbuf[1], kH2, kH1);
      commit();
    }
    wait_mma(3);
    for_chunks<kH2>(tz2, h, [&](int c0, float (&v)[16]) {
      float d[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float z = fmaf(v[j], F8 ? ssc2[c0 + j] : 1.f, sb2[c0 + j]);
        const float ez = ex2f(z * kexp);
        v[j] = z > 0.f ? z : al * (ez - 1.f);
        d[j] = z > 0.f ? 1.f : ez;
      }
      tmem_st16(tz2 + c0, d);  // CELU'(z2) for the backward
      if (F8) store_row16_e4m3(bufC, r, c0, v, q2);
      else store_row16(bufC, r, c0, v);
    });
    // ---------------- layer 3: z3 = h2 W3; energy and g3 = w4 CELU'(z3)
    if (!phase(0, -1)) break;
    if (tid == 0) {
      load_w(sp, 3, 1);                              // W3 (backward) -> wbuf[1]
      tc_fence_after();
      issue_gemm<F8>(mz3, bufC, wbuf[0], kH3, kH2);
      commit();
    }
    wait_mma(3);
    {
      float e = 0.f;
      for_chunks<kH3>(tz3, h, [&](int c0, float (&v)[16]) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float z = fmaf(v[j], F8 ? ssc3[c0 + j] : 1.f, sb3[c0 + j]);
          const float ww = sw4[c0 + j];
          const float ez = ex2f(z * kexp);
          e = fmaf(z > 0.f ? z : al * (ez - 1.f), ww, e);
          v[j] = ww * (z > 0.f ? 1.f : ez);
        }
        store_row16(bufC, r, c0, v);  // h2 no longer needed: the layer-3 MMA is done
      });
      sE[h * kTM + r] = e;
    }
    // ---------------- backward 3: g2' = g3 W3^T
    if (!phase(1, -1)) break;
    if (tid == 0) {
      load_w(sp, 4, 0);                              // W2 (backward) -> wbuf[0]
      tc_fence_after();
      issue_gemm<false>(mg2, bufC, wbuf[1], kH2, kH3);
      commit();
    }
    if (h == 0) {  // warps 0-3, one row per thread, while the MMA runs
      float e = *sb4;
#pragma unroll
      for (int g = 0; g < kG; ++g) e += sE[g * kTM + r];
      const bool valid = my_atom >= 0;
      const float ev = valid ? e : 0.f;
      if (accm) atomicAdd(&ws.Ei[row], ev);
      else ws.Ei[row] = ev;
      tile_energy_sums(ev, valid, my_sys, lane, io->energies);
    }
    wait_mma(3);
    for_chunks2<kH2>(tg2, tz2, h, [&](int c0, float (&g)[16], float (&d)[16]) {
#pragma unroll
      for (int j = 0; j < 16; ++j) g[j] *= d[j];
      store_row16(bufA, r, c0, g);  // the G tile is no longer needed
    });
    // ---------------- backward 2: g1' = g2 W2^T
    if (!phase(0, -1)) break;
    if (tid == 0) {
      load_w(sp, 5, 1);                              // W1 (backward) -> wbuf[1]
      tc_fence_after();
      issue_gemm<false>(mg1, bufA, wbuf[0], kH1, kH2);
      commit();
    }
    wait_mma(3);
    if (tid == 0 && has_next) {  // bufA and wbuf[0] are free: prefetch the next work item
      load_tile(next);
      load_wm(next_w, sp_next, 0, 0);
    }
    for_chunks2<kH1>(tg1, tz1, h, [&](int c0, float (&g)[16], float (&d)[16]) {
#pragma unroll
      for (int j = 0; j < 16; ++j) g[j] *= d[j];
      store_row16(bufB, r, c0, g);
    });
    // ---------------- backward 1: dE/dG = g1 W1^T
    if (!phase(1, -1)) break;
    if (tid == 0) {
      tc_fence_after();
      issue_gemm<false>(mdg, bufB, wbuf[1], D, kH1);
      commit();
    }
    wait_mma(3);
    if (tid == 0 && has_next) {  // next work item's layer 1 into [0,160), under the dE/dG epilogue
      wait0(2);
      wait0(0);
      if (*abort_flag == 0) {
        tc_fence_after();
        issue_gemm<F8>(mz1, bufA, wbuf[0], kH1, D);
        commit4();
        l1_issued = true;
      }
    }
    {  // staged through bufC (h2 / g3, read) and wbuf[1] (W1 backward, read)
      float4* stage = reinterpret_cast<float4*>(warp < 8 ? bufC + warp * 4096 : wbuf[1] + (warp - 8) * 4096);
      store_block_staged(tdg, h, lane, ws.dEdG + (size_t)(row0 + quarter * 32) * D, D, D, stage, accm);
    }
  }
  // on abort: give this CTA's outstanding copies and MMAs a bounded chance to land
  if (tid == 0 && *abort_flag) {
    for (int i = 0; i < 4; ++i)
      if (pend[i]) mbar_wait(&bars[i], ph[i]);
    if (pend4) mbar_wait(&bars[4], ph4);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Wide descriptors (three or more species, D > 128), BF16: the same network
// and epilogues, with the two products that involve D split into pieces that
// fit shared and tensor memory.
//
// * Layer 1, z1 = G W1: K one slab (64 features) at a time through four
//   stages; stage s takes G in bufA (s = 0, 1) or bufC (s = 2, 3) and W1^T in
//   wbuf[s / 2] (two 20 KB halves).  A slab's G and W1^T arrive on one barrier
//   (bars 10-13), and a stage is reloaded once the MMAs that read it have
//   completed (bars 14-17, waited by thread 0 only), so three slabs are in
//   flight while one is multiplied.
// * dE/dG = g1 W1^T: output columns in blocks of 128.  A block's weights are
//   the matching 128 rows of each of the three K slabs of the backward W1
//   image (three bulk copies).  Blocks alternate between wbuf[1] and wbuf[0];
//   the four 128-column quarters of tensor memory (all free after the g1
//   epilogue) take the accumulators in turn, and the next block's MMA runs
//   under this block's epilogue.  Blocks complete on bars 7 and 8, which
//   every thread waits on in turn.  The epilogue stages each warp's 32 rows x
//   32 columns in bufA or bufC (free once the backward MMAs that read g2 and
//   g3 are done) and writes whole 128-byte lines.
// The G tile is not fetched ahead of the tile, so layer 1 starts each tile
// with the latency of its first chunk.
// switch cases over the species counts with a wide descriptor (3..8)
#define NNP_WIDE_CASES(CALL) \
  case 3: CALL(3); break;    \
  case 4: CALL(4); break;    \
  case 5: CALL(5); break;    \
  case 6: CALL(6); break;    \
  case 7: CALL(7); break;    \
  default: CALL(8); break;
constexpr int kWideKC = 2;    // slabs of G that bufA and bufC each hold
constexpr int kWideNC = 128;  // dE/dG columns per block
constexpr int kWideBars = 18; // mbarriers of k_mlp_tc_wide

// g1out (ensembles): instead of the dE/dG blocks, each work item writes its
// g1 tile (the three swizzled slabs, as the MMA reads them) to slot
// tile * nm + member of g1out, and k_dedg_ens forms dE/dG from all members.
//
// F8: the three forward GEMMs in E4M3, as in k_mlp_tc: G arrives as E4M3
// (slabs of 128 columns; with D not a multiple of 32 the last MMA reads
// zeros past D in both operands), and the epilogues rescale by s_x s_W[n]
// and quantise h1 and h2 for the next layer; the backward stays BF16.
template <int D, bool F8>
__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_tc_wide(const EvalIO* __restrict__ io, DescParams P,
                                                       Workspace ws, const MlpTcWeights* __restrict__ Wts,
                                                       const MlpF32Weights* __restrict__ Wfs, int m0, int nm,
                                                       int accm, uint8_t* __restrict__ g1out) {
  constexpr int kBufA = kWideKC * kSlab;        // G chunk (stage 0), later g2
  constexpr int kBufB = slabs_of(kH1) * kSlab;  // h1, later g1
  constexpr int kBufC = slabs_of(kH2) * kSlab;  // G chunk (stage 1), h2, later g3
  constexpr int kWBuf = 48 * 1024;
  constexpr int kSl = F8 ? slabs8_of(D) : slabs_of(D);      // slabs of G and of W1^T
  constexpr int kNCB = (D + kWideNC - 1) / kWideNC;         // dE/dG blocks
  static_assert(D % 16 == 0 && D > kH2, "wide descriptor");
  static_assert(kBufA >= slabs_of(kH2) * kSlab && kBufC >= kWideKC * kSlab, "stage buffers");
  static_assert(2 * kH1 * 128 <= kWBuf && slabs_of(kH1) * kWideNC * 128 <= kWBuf, "weight buffers");
  constexpr int kNB = kH1 + kH2 + kH3 + kH3 + 1;  // b1 b2 b3 w4 b4

  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* bufA = sm;
  uint8_t* bufB = bufA + kBufA;
  uint8_t* bufC = bufB + kBufB;
  uint8_t* wbuf[2] = {bufC + kBufC, bufC + kBufC + kWBuf};
  // [0,1] weight copies, [3] MMAs, [4] layer 1 done, [7,8] dE/dG blocks,
  // [9] drain on abort, [10-13] layer-1 stage copies, [14-17] layer-1 stage
  // MMAs ([2], [5], [6] unused)
  uint64_t* bars = reinterpret_cast<uint64_t*>(wbuf[1] + kWBuf);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kWideBars);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  float* sE = reinterpret_cast<float*>(abort_flag + 1);  // [kG][kTM] partial energies
  float* sb = sE + kG * kTM;                             // [kNB] biases and w4 of the tile's species
  float* sb1 = sb;
  float* sb2 = sb1 + kH1;
  float* sb3 = sb2 + kH2;
  float* sw4 = sb3 + kH3;
  float* sb4 = sw4 + kH3;
  float* ssc = sb + kNB;  // FP8: [kH1 + kH2 + kH3] per-column dequantisation s_x s_W[n]
  float* ssc1 = ssc;
  float* ssc2 = ssc1 + kH1;
  float* ssc3 = ssc2 + kH2;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, h = warp >> 2;
  const int r = quarter * 32 + lane;
  const float al = P.celu_alpha, kexp = 1.4426950408889634f / P.celu_alpha;
  const int rows = ws.seg[P.S];
  const int ntiles = rows / kTM;

  if (tid == 0) {
    for (int i = 0; i < kWideBars; ++i) mbar_init(&bars[i], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lb = (uint32_t)(quarter * 32) << 16;
  const uint32_t tz1 = tmem + lb + 0, tz2 = tmem + lb + 160, tz3 = tmem + lb + 288, tg2 = tmem + lb + 384,
                 tg1 = tmem + lb + 160;
  const uint32_t mz1 = tmem + 0, mz2 = tmem + 160, mz3 = tmem + 288, mg2 = tmem + 384, mg1 = tmem + 160;
  // dE/dG block cb: accumulator in TMEM columns [128 (cb & 3), + 128); weights
  // in wbuf[1] (even cb, copies on bar 1) or wbuf[0] (odd cb, bar 0)
  auto dg_col = [](int cb) -> uint32_t { return (uint32_t)(cb & 3) * 128u; };
  auto dg_bar = [](int cb) -> int { return (cb & 1) ? 0 : 1; };
  auto dg_slab = [&](int cb, int k) -> uint8_t* { return wbuf[dg_bar(cb)] + (size_t)k * kWideNC * 128; };
  static_assert(8 * 4096 <= kBufA && 8 * 4096 <= kBufC, "dE/dG staging");
  static_assert((size_t)kBufB == kG1TileBytes, "g1 tile");

  uint32_t ph[4] = {0, 0, 0, 0};
  bool pend[4] = {false, false, false, false};
  uint32_t ph78[2] = {0, 0}, ph4 = 0;
  uint32_t phL[4] = {0, 0, 0, 0}, phM[4] = {0, 0, 0, 0};  // layer-1 stage copies / MMAs
  bool pendL[4] = {false, false, false, false};
  bool pend4 = false;

  const MlpTcWeights* cur_w = Wts + m0;  // the current work item's member
  const MlpF32Weights* cur_f = Wfs + m0;
  auto timeout = [&]() {
    *abort_flag = 1;
    atomicOr(&ws.flags[kFlagTimeout], 1);
  };
  auto load_w = [&](int sp, int which, int b) {  // a whole matrix (layers 2, 3 and backward 3, 2)
    constexpr int NWt[6] = {kH1, kH2, kH3, kH2, kH1, D};
    constexpr int KWt[6] = {D, kH1, kH2, kH3, kH2, kH1};
    const int bytes = (F8 && which < 3) ? mat8_bytes(NWt[which], KWt[which]) : mat_bytes(NWt[which], KWt[which]);
    mbar_expect_tx(&bars[b], (uint32_t)bytes);
    bulk_g2s(wbuf[b], cur_w->m[sp][which], (uint32_t)bytes, &bars[b]);
    pend[b] = true;
  };
  auto stage_g = [&](int st) { return (st < 2 ? bufA : bufC) + (size_t)(st & 1) * kSlab; };
  auto stage_w = [&](int st) { return wbuf[st >> 1] + (size_t)(st & 1) * kH1 * 128; };
  auto load_slab = [&](int t, int sp, int k) {  // G and W1^T slab k into stage k & 3
    const int st = k & 3;
    mbar_expect_tx(&bars[10 + st], (uint32_t)(kSlab + kH1 * 128));
    bulk_g2s(stage_g(st), reinterpret_cast<const uint8_t*>(ws.Gh) + (size_t)t * (F8 ? gh8_tile_bytes(D) : gh_tile_bytes(D)) +
                              (size_t)k * kSlab, (uint32_t)kSlab, &bars[10 + st]);
    bulk_g2s(stage_w(st), cur_w->m[sp][0] + (size_t)k * kH1 * 128, (uint32_t)(kH1 * 128), &bars[10 + st]);
    pendL[st] = true;
  };
  auto load_block = [&](int sp, int cb) {  // dE/dG block cb's W1 rows into its weight buffer
    const int n0 = cb * kWideNC, nc = min(kWideNC, D - n0), b = dg_bar(cb);
    const uint32_t bytes = (uint32_t)(nc * 128);
    mbar_expect_tx(&bars[b], (uint32_t)slabs_of(kH1) * bytes);
    for (int k = 0; k < slabs_of(kH1); ++k)
      bulk_g2s(dg_slab(cb, k), cur_w->m[sp][5] + (size_t)k * D * 128 + (size_t)n0 * 128, bytes, &bars[b]);
    pend[b] = true;
  };
  // D[128 x nc] = g1 (bufB, K = 160) x the block's weights (three slabs)
  auto issue_block = [&](int cb) {
    const int nc = min(kWideNC, D - cb * kWideNC);
    const uint32_t idesc = idesc_bf16(kTM, nc), a0 = smem_u32(bufB);
    for (int k = 0; k < kH1 / 16; ++k) {
      const uint32_t a = a0 + (uint32_t)(k >> 2) * kSlab + (uint32_t)(k & 3) * 32;
      const uint32_t b = smem_u32(dg_slab(cb, k >> 2)) + (uint32_t)(k & 3) * 32;
      mma_bf16(tmem + dg_col(cb), sw128_desc(a), sw128_desc(b), idesc, k > 0 ? 1u : 0u);
    }
  };
  auto commit = [&]() {
    mma_commit(&bars[3]);
    pend[3] = true;
  };
  auto wait0 = [&](int i) {  // thread 0: copies into buffer i have landed
    if (!pend[i]) return;
    if (mbar_wait(&bars[i], ph[i])) {
      ph[i] ^= 1u;
      pend[i] = false;
    } else {
      timeout();
    }
  };
  auto phase = [&](int i, int j) -> bool {
    tmem_wait_st();
    fence_proxy_async();
    tc_fence_before();
    if (tid == 0) {
      if (i >= 0) wait0(i);
      if (j >= 0) wait0(j);
    }
    __syncthreads();
    return *abort_flag == 0;
  };
  // every thread: MMAs committed to bar; idle: threads other than 0 back off
  // (layer 1, where thread 0 keeps streaming slabs while the others wait)
  auto wait_bar = [&](uint64_t* bar, uint32_t& p, bool idle = false) {
    if (warp == 0) __syncwarp();  // lanes 1-31 do not poll beside thread 0 while it issues
    if ((idle && tid != 0) ? mbar_wait_idle(bar, p) : mbar_wait(bar, p)) p ^= 1u;
    else timeout();
    tc_fence_after();
  };
  auto wait_mma = [&]() {
    wait_bar(&bars[3], ph[3]);
    if (tid == 0) pend[3] = false;
  };

  for (int wi = blockIdx.x; wi < ntiles * nm; wi += gridDim.x) {
    const int tile = wi / nm;  // member-minor, as in k_mlp_tc
    cur_w = Wts + m0 + wi % nm;
    cur_f = Wfs + m0 + wi % nm;
    const int row0 = tile * kTM;
    int sp = pos4_species(ws.pos4[row0]);
    if (!NNP_IN(sp, P.S, ws.flags)) sp = 0;
    const int row = row0 + r;
    const int my_atom = ws.row_atom[row];
    const int my_sys = ws.row_info[row];
    // FP8: z_l[n] = acc_l[n] * s_x s_W[n] + b_l[n]; q_l = 1 / s_{h_l} quantises h_l
    float q1 = 1.f, q2 = 1.f;
    if (F8) {
      const int* qs = ws.q8 + 8 * ((size_t)(m0 + wi % nm) * kMaxS + sp);  // this member's ranges
      if (tid == 0 && qs[0] == 0) atomicOr(&ws.flags[kFlagFp8Uncal], 1);  // the host calibrates and redoes
      const float sx0 = fp8_step(qs[0]), sx1 = fp8_step(qs[1]), sx2 = fp8_step(qs[2]);
      q1 = 1.f / sx1;
      q2 = 1.f / sx2;
      for (int i = tid; i < kH1 + kH2 + kH3; i += blockDim.x)
        ssc[i] = cur_w->wsc[sp][i] * (i < kH1 ? sx0 : (i < kH1 + kH2 ? sx1 : sx2));
    }
    for (int i = tid; i < kNB; i += blockDim.x) {
      float v;
      if (i < kH1) v = cur_f->b[sp][0][i];
      else if (i < kH1 + kH2) v = cur_f->b[sp][1][i - kH1];
      else if (i < kH1 + kH2 + kH3) v = cur_f->b[sp][2][i - kH1 - kH2];
      else if (i < kH1 + kH2 + 2 * kH3) v = cur_f->W[sp][3][i - kH1 - kH2 - kH3];
      else v = cur_f->b[sp][3][0];
      sb[i] = v;
    }
    if (!phase(-1, -1)) break;  // biases published; every buffer of the last tile is free
    // ---------------- layer 1: z1 = G W1, K one slab at a time through four stages
    if (tid == 0) {
      for (int k = 0; k < 4 && k < kSl; ++k) load_slab(tile, sp, k);
      for (int c = 0; c < kSl && *abort_flag == 0; ++c) {
        const int st = c & 3;
        if (mbar_wait(&bars[10 + st], phL[st])) {
          phL[st] ^= 1u;
          pendL[st] = false;
        } else {
          timeout();
          break;
        }
        tc_fence_after();
        // F8: K of the last slab rounded up to whole MMAs (zeros past D in both operands)
        const int kc = F8 ? min(128, (D - 128 * c + 31) / 32 * 32) : min(64, D - 64 * c);
        issue_gemm<F8>(mz1, stage_g(st), stage_w(st), kH1, kc, c > 0 ? 1u : 0u);
        if (c + 4 < kSl) mma_commit(&bars[14 + st]);  // stage st is reloaded once these MMAs are done
        if (c >= 1 && c + 3 < kSl) {                   // slab c - 1 has been read: its stage takes c + 3
          const int sq = (c - 1) & 3;
          if (mbar_wait(&bars[14 + sq], phM[sq])) phM[sq] ^= 1u;
          else timeout();
          if (*abort_flag == 0) load_slab(tile, sp, c + 3);
        }
      }
      mma_commit(&bars[4]);
      pend4 = true;
    }
    wait_bar(&bars[4], ph4, true);  // lanes 1-31 of warp 0 wait for thread 0 at a warp barrier
    if (tid == 0) {
      pend4 = false;
      if (*abort_flag == 0) {
        load_w(sp, 1, 1);  // W2^T -> wbuf[1]
        load_w(sp, 2, 0);  // W3^T -> wbuf[0]
      }
    }
    for_chunks<kH1>(tz1, h, [&](int c0, float (&v)[16]) {
      float d[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float z = fmaf(v[j], F8 ? ssc1[c0 + j] : 1.f, sb1[c0 + j]);
        const float ez = ex2f(z * kexp);
        v[j] = z > 0.f ? z : al * (ez - 1.f);
        d[j] = z > 0.f ? 1.f : ez;
      }
      tmem_st16(tz1 + c0, d);
      if (F8) store_row16_e4m3(bufB, r, c0, v, q1);
      else store_row16(bufB, r, c0, v);
    });
    // ---------------- layer 2: z2 = h1 W2
    if (!phase(1, -1)) break;
    if (tid == 0) {
      tc_fence_after();
      issue_gemm<F8>(mz2, bufB, wbuf[1], kH2, kH1);
      commit();
    }
    wait_mma();
    for_chunks<kH2>(tz2, h, [&](int c0, float (&v)[16]) {
      float d[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float z = fmaf(v[j], F8 ? ssc2[c0 + j] : 1.f, sb2[c0 + j]);
        const float ez = ex2f(z * kexp);
        v[j] = z > 0.f ? z : al * (ez - 1.f);
        d[j] = z > 0.f ? 1.f : ez;
      }
      tmem_st16(tz2 + c0, d);
      if (F8) store_row16_e4m3(bufC, r, c0, v, q2);
      else store_row16(bufC, r, c0, v);
    });
    // ---------------- layer 3: z3 = h2 W3; energy and g3 = w4 CELU'(z3)
    if (!phase(0, -1)) break;
    if (tid == 0) {
      load_w(sp, 3, 1);  // W3 (backward) -> wbuf[1]
      tc_fence_after();
      issue_gemm<F8>(mz3, bufC, wbuf[0], kH3, kH2);
      commit();
    }
    wait_mma();
    {
      float e = 0.f;
      for_chunks<kH3>(tz3, h, [&](int c0, float (&v)[16]) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float z = fmaf(v[j], F8 ? ssc3[c0 + j] : 1.f, sb3[c0 + j]);
          const float ww = sw4[c0 + j];
          const float ez = ex2f(z * kexp);
          e = fmaf(z > 0.f ? z : al * (ez - 1.f), ww, e);
          v[j] = ww * (z > 0.f ? 1.f : ez);
        }
        store_row16(bufC, r, c0, v);
      });
      sE[h * kTM + r] = e;
    }
    // ---------------- backward 3: g2' = g3 W3^T
    if (!phase(1, -1)) break;
    if (tid == 0) {
      load_w(sp, 4, 0);  // W2 (backward) -> wbuf[0]
      tc_fence_after();
      issue_gemm<false>(mg2, bufC, wbuf[1], kH2, kH3);
      commit();
    }
    if (h == 0) {
      float e = *sb4;
#pragma unroll
      for (int g = 0; g < kG; ++g) e += sE[g * kTM + r];
      const bool valid = my_atom >= 0;
      const float ev = valid ? e : 0.f;
      if (accm) atomicAdd(&ws.Ei[row], ev);
      else ws.Ei[row] = ev;
      tile_energy_sums(ev, valid, my_sys, lane, io->energies);
    }
    wait_mma();
    for_chunks2<kH2>(tg2, tz2, h, [&](int c0, float (&g)[16], float (&d)[16]) {
#pragma unroll
      for (int j = 0; j < 16; ++j) g[j] *= d[j];
      store_row16(bufA, r, c0, g);
    });
    // ---------------- backward 2: g1' = g2 W2^T
    if (!phase(0, -1)) break;
    if (tid == 0) {
      if (!g1out) load_block(sp, 0);  // dE/dG block 0 -> wbuf[1] (free since backward 3)
      tc_fence_after();
      issue_gemm<false>(mg1, bufA, wbuf[0], kH1, kH2);
      commit();
    }
    wait_mma();
    if (tid == 0 && kNCB > 1 && !g1out) load_block(sp, 1);  // wbuf[0] is free: block 1
    for_chunks2<kH1>(tg1, tz1, h, [&](int c0, float (&g)[16], float (&d)[16]) {
#pragma unroll
      for (int j = 0; j < 16; ++j) g[j] *= d[j];
      store_row16(bufB, r, c0, g);
    });
    // ---------------- backward 1: dE/dG = g1 W1^T in column blocks
    if (!phase(1, -1)) break;  // g1 written; block 0's weights have landed
    if (g1out) {  // ensemble: the g1 tile to its (tile, member) slot
      const uint4* src = reinterpret_cast<const uint4*>(bufB);
      uint4* dst = reinterpret_cast<uint4*>(g1out + ((size_t)tile * nm + wi % nm) * kG1TileBytes);
      for (int i = tid; i < (int)(kG1TileBytes / 16); i += blockDim.x) dst[i] = src[i];
      continue;  // the next item's first barrier comes before bufB is written again
    }
    if (tid == 0) {
      tc_fence_after();
      issue_block(0);
      mma_commit(&bars[7]);
    }
    bool ok = true;
    for (int cb = 0; cb < kNCB; ++cb) {
      const int q = cb & 1;  // block cb completes on bars[7 + q]
      const int n0 = cb * kWideNC, nc = min(kWideNC, D - n0);
      if (tid == 0 && cb + 1 < kNCB) {  // the next block's MMA runs under this block's epilogue
        wait0(dg_bar(cb + 1));
        if (*abort_flag == 0) {
          tc_fence_after();
          issue_block(cb + 1);
        }
        mma_commit(&bars[7 + (q ^ 1)]);
      }
      wait_bar(&bars[7 + q], ph78[q]);
      // block cb's weights have been read: its buffer takes block cb + 2
      if (tid == 0 && cb + 2 < kNCB && *abort_flag == 0) load_block(sp, cb + 2);
      float4* stage = reinterpret_cast<float4*>(warp < 8 ? bufA + warp * 4096 : bufC + (warp - 8) * 4096);
      store_block_staged(tmem + lb + dg_col(cb), h, lane, ws.dEdG + (size_t)(row0 + quarter * 32) * D + n0, D, nc,
                         stage, accm);
      if (!phase(-1, -1)) {  // this block's TMEM columns have been read before block cb + 4 reuses them
        ok = false;
        break;
      }
    }
    if (!ok) break;
  }
  // on abort: let this CTA's copies and MMAs land (bounded) before freeing TMEM
  if (tid == 0 && *abort_flag) {
    for (int i = 0; i < 2; ++i)
      if (pend[i]) mbar_wait(&bars[i], ph[i]);
    for (int i = 0; i < 4; ++i)
      if (pendL[i]) mbar_wait(&bars[10 + i], phL[i]);
    mma_commit(&bars[9]);
    mbar_wait(&bars[9], 0);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// dE/dG of an ensemble of wide networks, as one product over the members:
//   dE/dG[tile, block cb] = sum_m g1_m W1_m^T[:, block cb]  (K = 160 per member)
// Work items are (tile, 128-column block).  Thread 0 streams each member's g1
// tile (written by k_mlp_tc_wide) and W1 rows of the block through two 96 KB
// stages of shared memory and issues the MMAs, which accumulate in one TMEM
// block; the block is written once, as whole 128-byte lines
// (store_block_staged), so the members' shares meet in tensor memory instead
// of in L2 reductions, in a fixed order.  (Six 32 KB stages of single K slabs,
// with or without a separate producer thread, measured slower: 1.2-1.9x.)
constexpr int kEnsStage = 2 * (int)kG1TileBytes;  // one member's g1 tile and W1 block (48 KB each)
constexpr int kEnsBars = 5;                       // [0,1] stage copies, [2,3] stage MMAs, [4] block done
size_t smem_bytes_dedg() { return 1024 + 2 * (size_t)kEnsStage + kEnsBars * 8 + 16; }

template <int D>
__global__ void __launch_bounds__(kTcThreads, 1) k_dedg_ens(DescParams P, Workspace ws,
                                                    const MlpTcWeights* __restrict__ Wts,
                                                    const uint8_t* __restrict__ g1, int nm) {
  constexpr int kNCB = (D + kWideNC - 1) / kWideNC;
  constexpr uint32_t kCols = 128;
  static_assert(kTcThreads / 32 * 4096 <= kEnsStage, "epilogue staging");
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* stg[2] = {sm, sm + kEnsStage};
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * kEnsStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kEnsBars);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, h = warp >> 2;
  const int ntiles = ws.seg[P.S] / kTM;
  if (tid == 0) {
    for (int i = 0; i < kEnsBars; ++i) mbar_init(&bars[i], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lb = (uint32_t)(quarter * 32) << 16;
  uint32_t pc[2] = {0, 0}, pm[2] = {0, 0}, p4 = 0;
  bool pendc[2] = {false, false}, pendm[2] = {false, false};
  auto timeout = [&]() {
    *abort_flag = 1;
    atomicOr(&ws.flags[kFlagTimeout], 1);
  };
  for (int it = blockIdx.x; it < ntiles * kNCB; it += gridDim.x) {
    const int tile = it / kNCB, cb = it - tile * kNCB;
    const int row0 = tile * kTM, n0 = cb * kWideNC, nc = min(kWideNC, D - n0);
    if (tid == 0) {
      int sp = pos4_species(ws.pos4[row0]);
    if (!NNP_IN(sp, P.S, ws.flags)) sp = 0;
      const uint32_t wbytes = (uint32_t)(nc * 128);
      auto load = [&](int m, int st) {  // member m's g1 tile and W1 rows [n0, n0 + nc) into stage st
        mbar_expect_tx(&bars[st], (uint32_t)kG1TileBytes + (uint32_t)slabs_of(kH1) * wbytes);
        bulk_g2s(stg[st], g1 + ((size_t)tile * nm + m) * kG1TileBytes, (uint32_t)kG1TileBytes, &bars[st]);
        for (int k = 0; k < slabs_of(kH1); ++k)
          bulk_g2s(stg[st] + kG1TileBytes + (size_t)k * kWideNC * 128,
                   Wts[m].m[sp][5] + (size_t)k * D * 128 + (size_t)n0 * 128, wbytes, &bars[st]);
        pendc[st] = true;
      };
      load(0, 0);
      if (nm > 1) load(1, 1);
      const uint32_t idesc = idesc_bf16(kTM, nc);
      for (int m = 0; m < nm && *abort_flag == 0; ++m) {
        const int st = m & 1;
        if (mbar_wait(&bars[st], pc[st])) {
          pc[st] ^= 1u;
          pendc[st] = false;
        } else {
          timeout();
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(stg[st]), b0 = smem_u32(stg[st] + kG1TileBytes);
        for (int k = 0; k < kH1 / 16; ++k) {
          const uint32_t a = a0 + (uint32_t)(k >> 2) * kSlab + (uint32_t)(k & 3) * 32;
          const uint32_t b = b0 + (uint32_t)(k >> 2) * (uint32_t)(kWideNC * 128) + (uint32_t)(k & 3) * 32;
          mma_bf16(tmem, sw128_desc(a), sw128_desc(b), idesc, (m > 0 || k > 0) ? 1u : 0u);
        }
        if (m + 2 < nm) {  // stage st takes member m + 2 once these MMAs have read it
          mma_commit(&bars[2 + st]);
          pendm[st] = true;
          if (mbar_wait(&bars[2 + st], pm[st])) {
            pm[st] ^= 1u;
            pendm[st] = false;
          } else {
            timeout();
            break;
          }
          load(m + 2, st);
        }
      }
      mma_commit(&bars[4]);
    }
    if (warp == 0) __syncwarp();  // lanes 1-31 wait here, not polling beside thread 0
    if (mbar_wait_idle(&bars[4], p4)) p4 ^= 1u;
    else timeout();
    tc_fence_after();
    __syncthreads();
    if (*abort_flag) break;
    // every MMA is done: the stages take the epilogue's staging (4 KB per warp)
    float4* stage = reinterpret_cast<float4*>(sm + (size_t)warp * 4096);
    store_block_staged(tmem + lb, h, lane, ws.dEdG + (size_t)(row0 + quarter * 32) * D + n0, D, nc, stage, 0);
    fence_proxy_async();  // generic writes to the stages before the next item's copies
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  // on abort: let this CTA's copies and MMAs land (bounded) before freeing TMEM
  if (tid == 0 && *abort_flag) {
    for (int i = 0; i < 2; ++i) {
      if (pendc[i]) mbar_wait(&bars[i], pc[i]);
      if (pendm[i]) mbar_wait(&bars[2 + i], pm[i]);
    }
    mma_commit(&bars[4]);
    mbar_wait(&bars[4], p4);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ---------------------------------------------------------------------------
// Self-test of the bounded waits: a barrier that nothing completes.  Thread 0
// waits on it with the network kernel's own wait, gives up after limit_ns,
// raises the timeout flag and returns; the context stays usable.
__global__ void k_wait_selftest(int* flags, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_for(&bar, 0, limit_ns)) atomicOr(&flags[kFlagTimeout], 1);
}

void launch_wait_selftest(cudaStream_t st, int* flags, unsigned long long limit_ns) {
  k_wait_selftest<<<1, 32, 0, st>>>(flags, limit_ns);
}

// ---------------------------------------------------------------------------
// FP8 calibration: one warp per row runs the FP32 forward of layers 1-2 from
// the FP32 descriptor and raises the species' |max| of G, h1 and h2 (float
// bits, non-negative, so integer atomicMax orders them).  Rows are species
// sorted, so a warp flushes its running maxima only when the species changes.
__global__ void __launch_bounds__(256) k_fp8_calib(DescParams P, Workspace ws, MlpF32Weights Wf, int member) {
  __shared__ float xs[8][kMaxD], ys[8][kH1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int D = P.D, rows = ws.seg[P.S];
  const float al = P.celu_alpha, inv_al = 1.f / P.celu_alpha;
  float* x = xs[warp];
  float* y = ys[warp];
  int cur = -1;
  float m[3] = {0.f, 0.f, 0.f};
  auto flush = [&]() {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      float v = m[l];
      for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0 && cur >= 0) atomicMax(&ws.q8[8 * ((size_t)member * kMaxS + cur) + l], __float_as_int(v));
      m[l] = 0.f;
    }
  };
  for (int row = blockIdx.x * 8 + warp; row < rows; row += gridDim.x * 8) {
    if (ws.row_atom[row] < 0) continue;  // padding (warp-uniform)
    const int sp = pos4_species(ws.pos4[row]);
    if (sp != cur) {
      flush();
      cur = sp;
    }
    const float* g = ws.G + (size_t)row * D;
    __syncwarp();
    for (int k = lane; k < D; k += 32) {
      x[k] = g[k];
      m[0] = fmaxf(m[0], fabsf(g[k]));
    }
    __syncwarp();
    for (int j = lane; j < kH1; j += 32) {
      float z = Wf.b[sp][0][j];
      for (int k = 0; k < D; ++k) z = fmaf(x[k], Wf.W[sp][0][(size_t)k * kH1 + j], z);
      const float h = z > 0.f ? z : al * (expf(z * inv_al) - 1.f);
      y[j] = h;
      m[1] = fmaxf(m[1], fabsf(h));
    }
    __syncwarp();
    for (int j = lane; j < kH2; j += 32) {
      float z = Wf.b[sp][1][j];
      for (int k = 0; k < kH1; ++k) z = fmaf(y[k], Wf.W[sp][1][(size_t)k * kH2 + j], z);
      const float h = z > 0.f ? z : al * (expf(z * inv_al) - 1.f);
      m[2] = fmaxf(m[2], fabsf(h));
    }
  }
  flush();
}

// ---------------------------------------------------------------------------
// host side

namespace {

struct TcState {
  bool f8 = false;
  uint8_t* blob = nullptr;   // pre-swizzled weights, all members and species
  float* wsc = nullptr;      // FP8 per-column weight scales, all species
  size_t per_species = 0;
  size_t off[6] = {0, 0, 0, 0, 0, 0};
  std::vector<MlpTcWeights> wm;  // one set of image pointers per ensemble member
  MlpTcWeights* d_wm = nullptr;  // device copies of wm and of the context's FP32 sets (biases)
  MlpF32Weights* d_wf = nullptr;
};

// Byte offset of element (n, k) of a swizzled K-major [N][K] image with
// elements of esize bytes (2: BF16, 64 per slab row; 1: E4M3, 128).
inline size_t swz_off(int N, int n, int k, int esize) {
  const int per = 128 / esize;  // elements per 128-byte row of a slab
  const int slab = k / per, kk = k % per, ch = kk * esize / 16, e = kk * esize % 16;
  return (size_t)slab * N * 128 + (size_t)n * 128 + (size_t)((ch ^ (n & 7)) << 4) + e;
}

// BF16 image of a logical [N][K] matrix (value(n, k)).
template <class F>
void swizzle_into(uint8_t* dst, int N, int K, F value) {
  memset(dst, 0, (size_t)mat_bytes(N, K));
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < K; ++k) {
      __nv_bfloat16 h = __float2bfloat16(value(n, k));
      memcpy(dst + swz_off(N, n, k, 2), &h, 2);
    }
}

// E4M3 image of value(n, k) / s[n] with one scale per output column n,
// s[n] = max_k |value(n, k)| / 448 (1 for an all-zero column).
template <class F>
void swizzle_e4m3_into(uint8_t* dst, float* s, int N, int K, F value) {
  memset(dst, 0, (size_t)mat8_bytes(N, K));
  for (int n = 0; n < N; ++n) {
    float amax = 0.f;
    for (int k = 0; k < K; ++k) amax = std::max(amax, std::fabs(value(n, k)));
    s[n] = amax > 0.f ? amax / kE4M3Max : 1.f;
    for (int k = 0; k < K; ++k)
      dst[swz_off(N, n, k, 1)] = (uint8_t)__nv_cvt_float_to_fp8(value(n, k) / s[n], __NV_SATFINITE, __NV_E4M3);
  }
}

size_t smem_bytes(int D) {
  const int a = slabs_of(D > kH2 ? D : kH2) * kSlab, b = slabs_of(kH1) * kSlab, c = slabs_of(kH2) * kSlab;
  return 1024 + (size_t)a + b + c + 2 * 48 * 1024 + 5 * 8 + 8 + kG * kTM * 4 +
         (kH1 + kH2 + 2 * kH3 + 1) * 4 + (kH1 + kH2 + kH3) * 4 + 64;
}

template <int D, bool F8>
cudaError_t set_smem(size_t sm) {
  return cudaFuncSetAttribute(k_mlp_tc<D, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

size_t smem_bytes_wide() {
  return 1024 + (size_t)kWideKC * kSlab + slabs_of(kH1) * kSlab + slabs_of(kH2) * kSlab + 2 * 48 * 1024 +
         kWideBars * 8 + 8 + kG * kTM * 4 + (kH1 + kH2 + 2 * kH3 + 1) * 4 + (kH1 + kH2 + kH3) * 4 + 64;
}

template <int S>
cudaError_t set_smem_wide() {
  cudaError_t e = cudaFuncSetAttribute(k_mlp_tc_wide<desc_len(S), false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes_wide());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_tc_wide<desc_len(S), true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes_wide());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dedg_ens<desc_len(S)>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes_dedg());
  return e;
}

}  // namespace

int mlp_tc_init(nnp_ctx* ctx) {
  const bool f8 = ctx->cfg.precision == NNP_FP8;
  const int D = ctx->P.D;
  if (!f8 && D != 128 && D != 48 && D != desc_len(ctx->P.S))
    return ctx->fail(NNP_ERR_UNSUPPORTED, "the BF16 tensor-core network takes the standard descriptor");
  if (f8 && ctx->P.S < 2)
    return ctx->fail(NNP_ERR_UNSUPPORTED, "the FP8 tensor-core network needs at least 2 species (D >= 128)");
  TcState* st = new TcState();
  st->f8 = f8;
  const int NW[6] = {kH1, kH2, kH3, kH2, kH1, D};
  const int KW[6] = {D, kH1, kH2, kH3, kH2, kH1};
  size_t o = 0;
  for (int i = 0; i < 6; ++i) {
    st->off[i] = o;
    o += (size_t)((f8 && i < 3) ? mat8_bytes(NW[i], KW[i]) : mat_bytes(NW[i], KW[i]));
    o = (o + 1023) / 1024 * 1024;
  }
  st->per_species = o;
  ctx->tc = st;
  const int sets = ctx->n_members + (ctx->has_charges ? 1 : 0);  // ensemble, then the charge network
  const size_t images = (size_t)sets * ctx->P.S;
  cudaError_t e = cudaMalloc(&st->blob, o * images);
  if (e != cudaSuccess) {
    st->blob = nullptr;
    return ctx->cuda_fail(e, "cudaMalloc tensor-core weights");
  }
  cudaMemset(st->blob, 0, o * images);
  st->wm.assign((size_t)sets, MlpTcWeights{});
  for (int m = 0; m < sets; ++m)
    for (int s = 0; s < ctx->P.S; ++s)
      for (int i = 0; i < 6; ++i) st->wm[(size_t)m].m[s][i] = st->blob + o * ((size_t)m * ctx->P.S + s) + st->off[i];
  if (f8) {
    e = cudaMalloc(&st->wsc, sizeof(float) * (kH1 + kH2 + kH3) * ctx->P.S * sets);
    if (e != cudaSuccess) {
      st->wsc = nullptr;
      return ctx->cuda_fail(e, "cudaMalloc FP8 weight scales");
    }
    for (int m = 0; m < sets; ++m)
      for (int s = 0; s < ctx->P.S; ++s)
        st->wm[(size_t)m].wsc[s] = st->wsc + (size_t)(kH1 + kH2 + kH3) * ((size_t)m * ctx->P.S + s);
  }
  e = cudaMalloc(&st->d_wm, sizeof(MlpTcWeights) * sets);
  if (e == cudaSuccess) e = cudaMemcpy(st->d_wm, st->wm.data(), sizeof(MlpTcWeights) * sets, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&st->d_wf, sizeof(MlpF32Weights) * sets);
  if (e == cudaSuccess)
    e = cudaMemcpy(st->d_wf, ctx->wf32m.data(), sizeof(MlpF32Weights) * sets, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "weight tables");
  e = cudaMalloc(&ctx->b_q8, sizeof(int) * 8 * kMaxS * sets);
  if (e != cudaSuccess) {
    ctx->b_q8 = nullptr;
    return ctx->cuda_fail(e, "cudaMalloc FP8 scales");
  }
  cudaMemset(ctx->b_q8, 0, sizeof(int) * 8 * kMaxS * sets);
  const size_t sm = smem_bytes(D);
  if (f8 && D == 128) e = set_smem<128, true>(sm);
  else if (D == 128) e = set_smem<128, false>(sm);
  else if (D == 48) e = set_smem<48, false>(sm);
  else {
#define WSM(s) e = set_smem_wide<s>()
    switch (ctx->P.S) { NNP_WIDE_CASES(WSM) }
#undef WSM
  }
  if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaFuncSetAttribute(k_mlp_tc)");
  return NNP_OK;
}

int mlp_tc_set_weights(nnp_ctx* ctx, int member, int s, const float* hb) {
  TcState* st = static_cast<TcState*>(ctx->tc);
  if (!st) return ctx->fail(NNP_ERR_UNSUPPORTED, "tensor-core state missing");
  const int D = ctx->P.D;
  // host blob layout: W1 (D x 160) b1 W2 (160 x 128) b2 W3 (128 x 96) b3 W4 b4
  const float* W1 = hb;
  const float* W2 = W1 + (size_t)D * kH1 + kH1;
  const float* W3 = W2 + (size_t)kH1 * kH2 + kH2;
  std::vector<uint8_t> img(st->per_species, 0);
  auto w1t = [&](int n, int k) { return W1[(size_t)k * kH1 + n]; };
  auto w2t = [&](int n, int k) { return W2[(size_t)k * kH2 + n]; };
  auto w3t = [&](int n, int k) { return W3[(size_t)k * kH3 + n]; };
  std::vector<float> sw(kH1 + kH2 + kH3, 1.f);
  if (st->f8) {
    swizzle_e4m3_into(img.data() + st->off[0], sw.data(), kH1, D, w1t);
    swizzle_e4m3_into(img.data() + st->off[1], sw.data() + kH1, kH2, kH1, w2t);
    swizzle_e4m3_into(img.data() + st->off[2], sw.data() + kH1 + kH2, kH3, kH2, w3t);
  } else {
    swizzle_into(img.data() + st->off[0], kH1, D, w1t);
    swizzle_into(img.data() + st->off[1], kH2, kH1, w2t);
    swizzle_into(img.data() + st->off[2], kH3, kH2, w3t);
  }
  swizzle_into(img.data() + st->off[3], kH2, kH3, [&](int n, int k) { return W3[(size_t)n * kH3 + k]; });
  swizzle_into(img.data() + st->off[4], kH1, kH2, [&](int n, int k) { return W2[(size_t)n * kH2 + k]; });
  swizzle_into(img.data() + st->off[5], D, kH1, [&](int n, int k) { return W1[(size_t)n * kH1 + k]; });
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(st->blob + st->per_species * ((size_t)member * ctx->P.S + s), img.data(), st->per_species,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && st->f8) {
    // new weights: the weight scales of species s, and every activation range is re-calibrated
    e = cudaMemcpy(st->wsc + sw.size() * ((size_t)member * ctx->P.S + s), sw.data(), sizeof(float) * sw.size(),
                   cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ctx->b_q8, 0, sizeof(int) * 8 * kMaxS * ctx->n_members);
    ctx->fp8_calibrated = false;
    ctx->fp8_pass_done = false;
    for (int t = 0; t < kMaxS; ++t) ctx->fp8_seen[t] = false;
  }
  if (e != cudaSuccess) return ctx->cuda_fail(e, "upload tensor-core weights");
  return NNP_OK;
}

void mlp_tc_free(nnp_ctx* ctx) {
  TcState* st = static_cast<TcState*>(ctx->tc);
  if (ctx->b_q8) cudaFree(ctx->b_q8);
  ctx->b_q8 = nullptr;
  if (!st) return;
  if (st->blob) cudaFree(st->blob);
  if (st->wsc) cudaFree(st->wsc);
  if (st->d_wm) cudaFree(st->d_wm);
  if (st->d_wf) cudaFree(st->d_wf);
  delete st;
  ctx->tc = nullptr;
}

int launch_mlp_tc(nnp_ctx* ctx, cudaStream_t stream, long long rows, int m0, int nm, int accm, const EvalIO* io_o,
                  const Workspace* ws_o) {
  TcState* st = static_cast<TcState*>(ctx->tc);
  if (!st) return ctx->fail(NNP_ERR_UNSUPPORTED, "tensor-core state missing");
  const int D = ctx->P.D;
  const long long tiles = (rows + kTM - 1) / kTM;
  const int grid = (int)std::max<long long>(1, std::min<long long>(tiles * nm, ctx->num_sms));
  const Workspace w = ws_o ? *ws_o : ctx->workspace();
  const EvalIO* io = io_o ? io_o : ctx->d_io;
  const size_t sm = smem_bytes(D);
  const MlpTcWeights* tw = st->d_wm;
  const MlpF32Weights* fw = st->d_wf;
  if (st->f8 && D == 128)
    k_mlp_tc<128, true><<<grid, kTcThreads, sm, stream>>>(io, ctx->P, w, tw, fw, m0, nm, accm);
  else if (D == 128)
    k_mlp_tc<128, false><<<grid, kTcThreads, sm, stream>>>(io, ctx->P, w, tw, fw, m0, nm, accm);
  else if (D == 48)
    k_mlp_tc<48, false><<<grid, kTcThreads, sm, stream>>>(io, ctx->P, w, tw, fw, m0, nm, accm);
  else {
    const size_t smw = smem_bytes_wide();
    // an ensemble run side by side (all members, outputs added): g1 tiles,
    // then dE/dG as one product over the members
    uint8_t* g1 = (accm && m0 == 0 && nm == ctx->n_members && ctx->ens_wide()) ? ctx->b_g1 : nullptr;
#define WIDE(s)                                                                                           \
  if (st->f8) k_mlp_tc_wide<desc_len(s), true><<<grid, kTcThreads, smw, stream>>>(io, ctx->P, w, tw, fw, m0, \
                                                                                   nm, accm, g1);         \
  else k_mlp_tc_wide<desc_len(s), false><<<grid, kTcThreads, smw, stream>>>(io, ctx->P, w, tw, fw, m0, nm, accm, g1)
    switch (ctx->P.S) { NNP_WIDE_CASES(WIDE) }
#undef WIDE
    if (g1) {
      const long long items = tiles * ((D + kWideNC - 1) / kWideNC);
      const int gd = (int)std::max<long long>(1, std::min<long long>(items, ctx->num_sms));
      const size_t smd = smem_bytes_dedg();
#define DEDG(s) k_dedg_ens<desc_len(s)><<<gd, kTcThreads, smd, stream>>>(ctx->P, w, tw, g1, nm)
      switch (ctx->P.S) { NNP_WIDE_CASES(DEDG) }
#undef DEDG
    }
  }
  return NNP_OK;
}

int launch_fp8_calib(nnp_ctx* ctx, cudaStream_t stream, long long rows) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((rows + 7) / 8, 8ll * ctx->num_sms));
  for (int m = 0; m < ctx->n_members; ++m)  // every member's activation ranges
    k_fp8_calib<<<grid, 256, 0, stream>>>(ctx->P, ctx->workspace(), ctx->wf32m[(size_t)m], m);
  return NNP_OK;
}

}  // namespace nnp
