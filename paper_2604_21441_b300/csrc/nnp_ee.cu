// nnp_ee.cu -- electrostatic embedding (Methods, the nnpot interface: the
// model predicts in vacuo charges of the ML atoms, which interact with the MM
// point charges, and the MM atoms receive forces).
//
//   q_i   = charge network of species s_i on the descriptor G_i (a second
//           per-element network of the energy network's shape)
//   q'_i  = q_i - (sum_k q_k - Q) / n                  (total charge Q)
//   V_i   = k_e sum_J Q_J / |r_J - r_i|,  e_i = -grad_i V_i  (every MM charge J;
//           minimum image in an orthorhombic box)
//   E     = E_NNP + sum_i q'_i V_i
//   F_i  += q'_i e_i - (V_i - mean V) dq_i/dr            (second term through
//           dE/dG += (V_i - mean V) dq_i/dG and the descriptor backward)
//   F_J   = k_e Q_J sum_i q'_i (r_J - r_i) / |r_J - r_i|^3
//
// The pipeline runs, after the energy network: k_ee_prep (MM and ML
// coordinates as FP32 hi + lo pairs, accumulators zeroed, the charge pass's
// I/O block), k_ee_potential, the charge network with its outputs redirected,
// k_ee_combine; after the descriptor backward: k_ee_finish, k_ee_mm_forces.
// Displacements are (hi_J - hi_i) + (lo_J - lo_i) in FP32: the hi difference
// rounds relative to the displacement, not to the coordinates, so pairs are
// good to about 1e-7 relative without the FP64 pipe.  Potentials and fields
// are summed in FP32 over a chunk of MM charges and in FP64 across chunks.
#include "nnp_host.h"

namespace nnp {

namespace {

constexpr double kCoulomb = 14.3996454784;  // e^2 / (4 pi eps0) in eV A
constexpr int kEeThreads = 128;             // ML atoms per potential block, MM atoms per force block
constexpr int kEeTile = 128;                // charges staged in shared memory per step

int ee_grid(long long items, int per_block, int cap) {
  long long g = (items + per_block - 1) / per_block;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

__device__ __forceinline__ void split2(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// d = (b - a) with minimum image, from hi/lo parts of coordinates wrapped
// into [0, L) (so |d| < L and one shift at most; selects, no rounding)
__device__ __forceinline__ float3 disp(float4 ah, float4 al, float4 bh, float4 bl, const EeIO& e) {
  float d[3] = {(bh.x - ah.x) + (bl.x - al.x), (bh.y - ah.y) + (bl.y - al.y), (bh.z - ah.z) + (bl.z - al.z)};
  if (e.periodic) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float half = 0.5f * e.Lhi[c];
      const float s = d[c] > half ? 1.f : (d[c] < -half ? -1.f : 0.f);
      d[c] = fmaf(-s, e.Llo[c], fmaf(-s, e.Lhi[c], d[c]));
    }
  }
  return make_float3(d[0], d[1], d[2]);
}

// x wrapped into [0, L) in FP64 (periodic axes), then split into hi + lo
__device__ __forceinline__ void wrap_split(double x, int c, const EeIO& e, float& hi, float& lo) {
  if (e.periodic) {
    x -= e.L[c] * floor(x * e.invL[c]);
    if (x < 0.0) x += e.L[c];
    if (x >= e.L[c]) x -= e.L[c];
  }
  split2(x, hi, lo);
}

}  // namespace

__global__ void k_ee_prep(const EvalIO* __restrict__ io, EvalIO* __restrict__ io_q, const EeIO* __restrict__ ee) {
  const EeIO& e = *ee;
  const long long n = io->n_atoms, m = e.n_mm;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  if (tid == 0) {
    *io_q = *io;
    io_q->energies = e.sums;  // the charge pass's per-system sum (not used)
    e.sums[0] = 0.0;
    e.sums[1] = 0.0;          // sum_i V_i
    e.sums[2] = 0.0;          // sum_i q_i, in FP64 over the stored charges
  }
  for (long long j = tid; j < m; j += stride) {
    float h[3], l[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) wrap_split(e.mm_pos[3 * j + c], c, e, h[c], l[c]);
    e.mm_hi[j] = make_float4(h[0], h[1], h[2], (float)e.mm_q[j]);
    e.mm_lo[j] = make_float4(l[0], l[1], l[2], 0.f);
  }
  for (long long a = tid; a < n; a += stride) {
    float h[3], l[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) wrap_split(io->pos[3 * a + c], c, e, h[c], l[c]);
    e.ml_hi[a] = make_float4(h[0], h[1], h[2], 0.f);
    e.ml_lo[a] = make_float4(l[0], l[1], l[2], 0.f);
    e.V[a] = 0.0;
    e.field[3 * a] = 0.0;
    e.field[3 * a + 1] = 0.0;
    e.field[3 * a + 2] = 0.0;
  }
}

// Block (x: 128 ML atoms, y: a chunk of MM charges).  Each thread sums its ML
// atom's potential and field over the chunk in FP32, then adds in FP64.
__global__ void __launch_bounds__(kEeThreads) k_ee_potential(const EvalIO* __restrict__ io,
                                                             const EeIO* __restrict__ ee) {
  __shared__ float4 sh[kEeTile], sl[kEeTile];
  const EeIO& e = *ee;
  const long long n = io->n_atoms, m = e.n_mm;
  const long long chunk = (m + gridDim.y - 1) / gridDim.y;
  const long long j0 = (long long)blockIdx.y * chunk, j1 = j0 + chunk < m ? j0 + chunk : m;
  const long long a = (long long)blockIdx.x * kEeThreads + threadIdx.x;
  const bool live = a < n;
  const float4 ah = live ? e.ml_hi[a] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 al = live ? e.ml_lo[a] : make_float4(0.f, 0.f, 0.f, 0.f);
  float v = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
  for (long long t0 = j0; t0 < j1; t0 += kEeTile) {
    const int nt = (int)(j1 - t0 < kEeTile ? j1 - t0 : kEeTile);
    __syncthreads();
    if (threadIdx.x < nt) {
      sh[threadIdx.x] = e.mm_hi[t0 + threadIdx.x];
      sl[threadIdx.x] = e.mm_lo[t0 + threadIdx.x];
    }
    __syncthreads();
    if (live) {
#pragma unroll 4
      for (int k = 0; k < nt; ++k) {
        const float3 d = disp(ah, al, sh[k], sl[k], e);
        const float r2 = fmaf(d.z, d.z, fmaf(d.y, d.y, d.x * d.x));
        const float ir = rsqrtf(r2);
        const float qr = sh[k].w * ir;  // Q / r
        const float qr3 = qr * ir * ir;
        v += qr;
        fx = fmaf(-qr3, d.x, fx);  // e = -grad_i V = -sum Q (r_J - r_i) / r^3
        fy = fmaf(-qr3, d.y, fy);
        fz = fmaf(-qr3, d.z, fz);
      }
    }
  }
  if (live && j1 > j0) {
    atomicAdd(&e.V[a], kCoulomb * (double)v);
    atomicAdd(&e.field[3 * a], kCoulomb * (double)fx);
    atomicAdd(&e.field[3 * a + 1], kCoulomb * (double)fy);
    atomicAdd(&e.field[3 * a + 2], kCoulomb * (double)fz);
  }
  // sum of V over the block, then one add per block (one address is shared by all blocks)
  __shared__ double red[kEeThreads / 32];
  double vs = (live && j1 > j0) ? kCoulomb * (double)v : 0.0;
  for (int o = 16; o; o >>= 1) vs += __shfl_xor_sync(0xffffffffu, vs, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vs;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kEeThreads / 32; ++k) t += red[k];
    if (t != 0.0) atomicAdd(&e.sums[1], t);
  }
}

// dE/dG of row r += (V_i - mean V) dq_i/dG (i the row's atom), and the raw
// charge of the atom in input order.
__global__ void k_ee_combine(const EvalIO* __restrict__ io, const EeIO* __restrict__ ee, int D, Workspace ws) {
  const EeIO& e = *ee;
  const long long n = io->n_atoms;
  const int rows = ws.seg[e.S];
  const double vbar = e.sums[1] / (double)n;
  const long long total = (long long)rows * D;
  double qsum = 0.0;  // this thread's raw charges; one add per block below
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(t / D), f = (int)(t - (long long)row * D);
    const int a = ws.row_atom[row];
    if (a < 0) continue;
    const float c = (float)(e.V[a] - vbar);
    ws.dEdG[t] = fmaf(c, e.dqdG[t], ws.dEdG[t]);
    if (f == 0) {
      const double q = (double)e.q_rows[row];
      e.q_atom[a] = q;
      qsum += q;
    }
  }
  __shared__ double red[32];
  for (int o = 16; o; o >>= 1) qsum += __shfl_xor_sync(0xffffffffu, qsum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = qsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    if (t != 0.0) atomicAdd(&e.sums[2], t);
  }
}

// After the descriptor backward: q', the embedding energy, the direct ML forces.
__global__ void k_ee_finish(const EvalIO* __restrict__ io, const EeIO* __restrict__ ee) {
  __shared__ double red[32];
  const EeIO& e = *ee;
  const long long n = io->n_atoms;
  const double shift = (e.sums[2] - e.Q) / (double)n;
  double part = 0.0;
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < n;
       a += (long long)gridDim.x * blockDim.x) {
    const double q = e.q_atom[a] - shift;
    e.q_out[a] = q;
    part += q * e.V[a];
    double* F = io->forces + 3 * a;
    F[0] += q * e.field[3 * a];
    F[1] += q * e.field[3 * a + 1];
    F[2] += q * e.field[3 * a + 2];
  }
  for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    atomicAdd(&io->energies[0], s);
  }
}

// One thread per MM charge: F_J = k_e Q_J sum_i q'_i (r_J - r_i) / r^3.
__global__ void __launch_bounds__(kEeThreads) k_ee_mm_forces(const EvalIO* __restrict__ io,
                                                             const EeIO* __restrict__ ee) {
  __shared__ float4 sh[kEeTile], sl[kEeTile];
  const EeIO& e = *ee;
  const long long n = io->n_atoms, m = e.n_mm;
  const long long j = (long long)blockIdx.x * kEeThreads + threadIdx.x;
  const bool live = j < m;
  const float4 bh = live ? e.mm_hi[j] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 bl = live ? e.mm_lo[j] : make_float4(0.f, 0.f, 0.f, 0.f);
  float fx = 0.f, fy = 0.f, fz = 0.f;
  for (long long t0 = 0; t0 < n; t0 += kEeTile) {
    const int nt = (int)(n - t0 < kEeTile ? n - t0 : kEeTile);
    __syncthreads();
    if (threadIdx.x < nt) {
      float4 h = e.ml_hi[t0 + threadIdx.x];
      h.w = (float)e.q_out[t0 + threadIdx.x];
      sh[threadIdx.x] = h;
      sl[threadIdx.x] = e.ml_lo[t0 + threadIdx.x];
    }
    __syncthreads();
    if (live) {
#pragma unroll 4
      for (int k = 0; k < nt; ++k) {
        const float3 d = disp(sh[k], sl[k], bh, bl, e);  // r_J - r_i
        const float r2 = fmaf(d.z, d.z, fmaf(d.y, d.y, d.x * d.x));
        const float ir = rsqrtf(r2);
        const float s = sh[k].w * ir * ir * ir;
        fx = fmaf(s, d.x, fx);
        fy = fmaf(s, d.y, fy);
        fz = fmaf(s, d.z, fz);
      }
    }
  }
  if (live) {
    const double kq = kCoulomb * (double)bh.w;
    e.mm_forces[3 * j] = kq * fx;
    e.mm_forces[3 * j + 1] = kq * fy;
    e.mm_forces[3 * j + 2] = kq * fz;
  }
}

}  // namespace nnp

// ---------------------------------------------------------------------------
// host side

using namespace nnp;

int nnp_ctx::launch_ee_pre(long long rows, const Workspace& w, int& launches) {
  const int nsm = num_sms;
  const long long n = ee_n_ml, m = ee_n_mm;
  k_ee_prep<<<ee_grid(std::max(n, m), 256, nsm * 4), 256, 0, stream>>>(d_io, d_io_q, d_ee); ++launches;
  const int bx = (int)((n + kEeThreads - 1) / kEeThreads);
  long long by = (8LL * nsm + bx - 1) / bx;  // enough blocks to hide the pair loop's latency
  by = std::max(1LL, std::min(by, (m + kEeTile - 1) / kEeTile));
  k_ee_potential<<<dim3(bx, (unsigned)by), kEeThreads, 0, stream>>>(d_io, d_ee); ++launches;
  // charge network: per-row outputs and dq/dG into the embedding's buffers
  Workspace wq = w;
  wq.Ei = b_ee_qrows;
  wq.dEdG = b_ee_dqdG;
  const int qm = n_members;  // the charge network's weight set follows the ensemble
  if (cfg.precision == NNP_FP32) {
    const int g_tiles = (int)std::min<long long>(rows / 64, (long long)nsm);
    launch_mlp_f32(std::max(1, g_tiles), stream, d_io_q, P, wq, wf32m[(size_t)qm], 0);
  } else {
    int rc = launch_mlp_tc(this, stream, rows, qm, 1, 0, d_io_q, &wq);
    if (rc) return rc;
  }
  ++launches;
  k_ee_combine<<<ee_grid(rows * P.D, 256, nsm * 8), 256, 0, stream>>>(d_io, d_ee, P.D, w); ++launches;
  return NNP_OK;
}

void nnp_ctx::launch_ee_post(int& launches) {
  const int nsm = num_sms;
  k_ee_finish<<<ee_grid(ee_n_ml, 256, nsm), 256, 0, stream>>>(d_io, d_ee); ++launches;
  k_ee_mm_forces<<<ee_grid(ee_n_mm, kEeThreads, 1 << 30), kEeThreads, 0, stream>>>(d_io, d_ee);
  ++launches;
}

extern "C" int nnp_set_charge_weights(nnp_ctx* ctx, int32_t species, const float* const W[4],
                                      const float* const b[4]) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (!ctx->has_charges) return ctx->fail(NNP_ERR_UNSUPPORTED, "context created without NNP_FLAG_CHARGES");
  if (species < 0 || species >= ctx->P.S) return ctx->fail(NNP_ERR_INVALID_ARG, "species index %d", species);
  if (!W || !b) return ctx->fail(NNP_ERR_INVALID_ARG, "null weight arrays");
  for (int l = 0; l < 4; ++l)
    if (!W[l] || !b[l]) return ctx->fail(NNP_ERR_INVALID_ARG, "null weight or bias of layer %d", l);
  return ctx->set_weights(ctx->n_members, species, W, b);
}

extern "C" int nnp_eval_ee(nnp_ctx* ctx, int64_t n, const double* pos, const int32_t* Z, const double* box,
                           int64_t n_mm, const double* mm_pos, const double* mm_q, double total_charge,
                           double* energy, double* forces, double* mm_forces, double* charges) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (!ctx->has_charges) return ctx->fail(NNP_ERR_UNSUPPORTED, "context created without NNP_FLAG_CHARGES");
  if (n <= 0) return ctx->fail(NNP_ERR_INVALID_ARG, "n must be positive");
  if (n_mm < 0 || (n_mm > 0 && (!mm_pos || !mm_q))) return ctx->fail(NNP_ERR_INVALID_ARG, "null MM arrays");
  if (!std::isfinite(total_charge)) return ctx->fail(NNP_ERR_INVALID_ARG, "non-finite total charge");
  if (!ctx->charges_ready()) return ctx->fail(NNP_ERR_NO_WEIGHTS, "charge-network weights missing for some species");
  int periodic = 0;
  float Lhi[3] = {0.f, 0.f, 0.f}, Llo[3] = {0.f, 0.f, 0.f};
  double Ld[3] = {0.0, 0.0, 0.0}, invL[3] = {0.0, 0.0, 0.0};
  if (box) {
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        if (r != c && box[3 * r + c] != 0.0)
          return ctx->fail(NNP_ERR_UNSUPPORTED, "the embedding takes orthorhombic boxes");
    periodic = 1;
    for (int c = 0; c < 3; ++c) {
      const double L = box[4 * c];
      if (!(L > 0.0)) return ctx->fail(NNP_ERR_INVALID_ARG, "box edge %d is %g", c, L);
      Lhi[c] = (float)L;
      Llo[c] = (float)(L - (double)Lhi[c]);
      Ld[c] = L;
      invL[c] = 1.0 / L;
    }
  }
  const long long m = std::max<long long>(n_mm, 1);
  cudaError_t e = ctx->ee_reserve(n, m);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "embedding buffers");
  EeIO& h = *ctx->h_ee;
  h.periodic = periodic;
  for (int c = 0; c < 3; ++c) {
    h.Lhi[c] = Lhi[c];
    h.Llo[c] = Llo[c];
    h.L[c] = Ld[c];
    h.invL[c] = invL[c];
  }
  cudaStream_t st = ctx->stream;
  const bool dev_mmx = n_mm == 0 || nnp_ctx::is_device(mm_pos), dev_mmq = n_mm == 0 || nnp_ctx::is_device(mm_q);
  if (!dev_mmx) e = cudaMemcpyAsync(ctx->b_ee_mmpos, mm_pos, sizeof(double) * 3 * n_mm, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !dev_mmq)
    e = cudaMemcpyAsync(ctx->b_ee_mmq, mm_q, sizeof(double) * n_mm, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "copy MM charges");
  const bool dev_mmF = mm_forces && nnp_ctx::is_device(mm_forces);
  const bool dev_q = charges && nnp_ctx::is_device(charges);
  h.mm_pos = dev_mmx ? mm_pos : ctx->b_ee_mmpos;
  h.mm_q = dev_mmq ? mm_q : ctx->b_ee_mmq;
  h.n_mm = n_mm;
  h.Q = total_charge;
  h.S = ctx->P.S;
  h.mm_forces = dev_mmF ? mm_forces : ctx->b_ee_mmF;
  h.q_out = dev_q ? charges : ctx->b_ee_qout;
  e = cudaMemcpyAsync(ctx->d_ee, &h, sizeof(EeIO), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "embedding parameters");
  ctx->ee_mode = true;
  ctx->ee_n_ml = n;
  ctx->ee_n_mm = n_mm;
  int64_t off[2] = {0, n};
  int rc = ctx->evaluate(1, off, pos, Z, box, energy, forces, true);
  ctx->ee_mode = false;
  if (rc) return rc;
  if (mm_forces && !dev_mmF && n_mm > 0)
    e = cudaMemcpy(mm_forces, ctx->b_ee_mmF, sizeof(double) * 3 * n_mm, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && charges && !dev_q)
    e = cudaMemcpy(charges, ctx->b_ee_qout, sizeof(double) * n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "copy embedding results");
  return NNP_OK;
}

// Embedding buffers for n ML atoms and m MM charges (grown on demand).
cudaError_t nnp_ctx::ee_reserve(long long n, long long m) {
  cudaError_t e = cudaSuccess;
  bool moved = false;
  auto grow = [&](auto*& p, size_t need, size_t elem) {
    if (e != cudaSuccess) return;
    if (p) cudaFree(p);
    p = nullptr;
    e = cudaMalloc(reinterpret_cast<void**>(&p), elem * need);
    moved = true;
  };
  if (!h_ee) {
    e = cudaMallocHost(&h_ee, sizeof(EeIO));
    if (e == cudaSuccess) e = cudaMalloc(&d_ee, sizeof(EeIO));
    if (e == cudaSuccess) e = cudaMalloc(&d_io_q, sizeof(EvalIO));
    if (e == cudaSuccess) e = cudaMalloc(&b_ee_sums, sizeof(double) * 4);
    if (e != cudaSuccess) return e;
    memset(h_ee, 0, sizeof(EeIO));
  }
  const long long rows = n + (long long)kTileRows * P.S;
  if ((size_t)n > c_ee_n || (size_t)rows > c_ee_rows || (size_t)m > c_ee_m) {
    e = cudaStreamSynchronize(stream);  // nothing in flight may use a buffer that is replaced
    if (e != cudaSuccess) return e;
  }
  if ((size_t)n > c_ee_n) {
    grow(b_ee_mlhi, n, sizeof(float4));
    grow(b_ee_mllo, n, sizeof(float4));
    grow(b_ee_V, n, sizeof(double));
    grow(b_ee_field, 3 * n, sizeof(double));
    grow(b_ee_qatom, n, sizeof(double));
    grow(b_ee_qout, n, sizeof(double));
    if (e != cudaSuccess) return e;
    c_ee_n = n;
  }
  if ((size_t)rows > c_ee_rows) {
    grow(b_ee_qrows, rows, sizeof(float));
    grow(b_ee_dqdG, (size_t)rows * P.D, sizeof(float));
    if (e != cudaSuccess) return e;
    c_ee_rows = rows;
  }
  if ((size_t)m > c_ee_m) {
    grow(b_ee_mmhi, m, sizeof(float4));
    grow(b_ee_mmlo, m, sizeof(float4));
    grow(b_ee_mmF, 3 * m, sizeof(double));
    grow(b_ee_mmpos, 3 * m, sizeof(double));
    grow(b_ee_mmq, m, sizeof(double));
    if (e != cudaSuccess) return e;
    c_ee_m = m;
  }
  EeIO& h = *h_ee;
  h.mm_hi = b_ee_mmhi;
  h.mm_lo = b_ee_mmlo;
  h.ml_hi = b_ee_mlhi;
  h.ml_lo = b_ee_mllo;
  h.V = b_ee_V;
  h.field = b_ee_field;
  h.q_rows = b_ee_qrows;
  h.dqdG = b_ee_dqdG;
  h.q_atom = b_ee_qatom;
  h.sums = b_ee_sums;
  if (moved) invalidate_graph();  // the charge pass's buffers are baked into the graph
  return cudaSuccess;
}
