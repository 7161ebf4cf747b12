// nnp_mlmm.cu -- ML/MM mechanical embedding around the NNP evaluation
// (Sec. Methods, "The nnpot Interface", link-atom equation).
//
// The ML group (an index set of a larger system) plus one link atom per cut
// ML-MM bond form the subsystem the NNP sees.  A link atom sits on the bond at
// a fixed distance d from its ML atom,
//   r_L = r_ML + d u,  u = R / |R|,  R = r_MM - r_ML  (minimum image in the box),
// and carries the user's link type (hydrogen by default).  Its force F_L goes
// back to the two bonded atoms by the chain rule:
//   dr_L/dr_MM = (d / |R|) (I - u u^T),   dr_L/dr_ML = I - dr_L/dr_MM,
// so F_MM += (d / |R|) (F_L - u (u . F_L)) and F_ML += F_L - that share.
//
// Device flow on the context's stream: validation of device-resident index
// sets, gather (subsystem positions and species), the ordinary evaluation on
// device buffers, scatter (ML forces by index, then the link shares).
#include <cstring>
#include <vector>

#include "nnp_host.h"

namespace nnp {
namespace {

// minimum image of a displacement in an orthorhombic box (L <= 0: open)
__device__ __forceinline__ double min_image(double x, double L) {
  return L > 0.0 ? x - L * nearbyint(x / L) : x;
}

// validation of device-resident index sets (host-resident ones are checked on
// the host): bit 1 index out of range, 2 repeated group index, 4 link atom
// outside the group, 8 link MM atom inside it, 16 link distance <= 0, 32 a
// zero-length bond (set by the gather)
enum { kBadRange = 1, kBadRepeat = 2, kBadLinkMl = 4, kBadLinkMm = 8, kBadDist = 16, kBadBond = 32 };

__global__ void k_mlmm_mark(const int64_t* __restrict__ ml_index, long long n_ml, long long n_total,
                            int* __restrict__ mark, int* __restrict__ bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_ml; k += stride) {
    const long long a = ml_index[k];
    if (a < 0 || a >= n_total) {
      atomicOr(bad, kBadRange);
      continue;
    }
    if (atomicExch(&mark[a], 1)) atomicOr(bad, kBadRepeat);
  }
}

__global__ void k_mlmm_check_links(const int64_t* __restrict__ link_ml, const int64_t* __restrict__ link_mm,
                                   const double* __restrict__ link_d, int n_link, long long n_total,
                                   const int* __restrict__ mark, int* __restrict__ bad) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n_link; l += gridDim.x * blockDim.x) {
    const long long i = link_ml[l], j = link_mm[l];
    if (i < 0 || i >= n_total || j < 0 || j >= n_total) {
      atomicOr(bad, kBadRange);
      continue;
    }
    if (!mark[i]) atomicOr(bad, kBadLinkMl);
    if (mark[j]) atomicOr(bad, kBadLinkMm);
    if (!(link_d[l] > 0.0)) atomicOr(bad, kBadDist);
  }
}

// indices out of range (flagged above) are skipped, so no access leaves the arrays
__global__ void k_mlmm_gather(const double* __restrict__ pos, const int32_t* __restrict__ Z,
                              const int64_t* __restrict__ ml_index, long long n_ml, long long n_total,
                              const int64_t* __restrict__ link_ml, const int64_t* __restrict__ link_mm,
                              const double* __restrict__ link_d, int n_link, int link_Z, double3 L,
                              double* __restrict__ sub_pos, int32_t* __restrict__ sub_Z,
                              int* __restrict__ bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_ml + n_link; k += stride) {
    if (k < n_ml) {
      long long a = ml_index[k];
      if (a < 0 || a >= n_total) a = 0;
      sub_pos[3 * k] = pos[3 * a];
      sub_pos[3 * k + 1] = pos[3 * a + 1];
      sub_pos[3 * k + 2] = pos[3 * a + 2];
      sub_Z[k] = Z[a];
    } else {
      const int l = (int)(k - n_ml);
      long long i = link_ml[l], j = link_mm[l];
      if (i < 0 || i >= n_total || j < 0 || j >= n_total) i = j = 0;
      const double Rx = min_image(pos[3 * j] - pos[3 * i], L.x);
      const double Ry = min_image(pos[3 * j + 1] - pos[3 * i + 1], L.y);
      const double Rz = min_image(pos[3 * j + 2] - pos[3 * i + 2], L.z);
      const double R = sqrt(Rx * Rx + Ry * Ry + Rz * Rz);
      if (!(R > 0.0)) atomicOr(bad, kBadBond);
      const double s = R > 0.0 ? link_d[l] / R : 0.0;
      sub_pos[3 * k] = pos[3 * i] + s * Rx;
      sub_pos[3 * k + 1] = pos[3 * i + 1] + s * Ry;
      sub_pos[3 * k + 2] = pos[3 * i + 2] + s * Rz;
      sub_Z[k] = link_Z;
    }
  }
}

// the ML atoms' own forces (distinct indices) into the zeroed full-system array
__global__ void k_mlmm_scatter_ml(const double* __restrict__ sub_F, const int64_t* __restrict__ ml_index,
                                  long long n_ml, double* __restrict__ F) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_ml; k += stride) {
    const long long a = ml_index[k];
    F[3 * a] = sub_F[3 * k];
    F[3 * a + 1] = sub_F[3 * k + 1];
    F[3 * a + 2] = sub_F[3 * k + 2];
  }
}

// link shares, thread per link; FP64 atomic adds (an atom that several links
// share may see its sums in another order from call to call, in the last bit)
__global__ void k_mlmm_links(const double* __restrict__ pos, const double* __restrict__ sub_F, long long n_ml,
                             const int64_t* __restrict__ link_ml, const int64_t* __restrict__ link_mm,
                             const double* __restrict__ link_d, int n_link, double3 L, double* __restrict__ F) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n_link; l += gridDim.x * blockDim.x) {
    const long long i = link_ml[l], j = link_mm[l];
    const double Rx = min_image(pos[3 * j] - pos[3 * i], L.x);
    const double Ry = min_image(pos[3 * j + 1] - pos[3 * i + 1], L.y);
    const double Rz = min_image(pos[3 * j + 2] - pos[3 * i + 2], L.z);
    const double R = sqrt(Rx * Rx + Ry * Ry + Rz * Rz);
    if (!(R > 0.0)) continue;  // reported by the gather
    const double ux = Rx / R, uy = Ry / R, uz = Rz / R;
    const double s = link_d[l] / R;
    const double fx = sub_F[3 * (n_ml + l)], fy = sub_F[3 * (n_ml + l) + 1], fz = sub_F[3 * (n_ml + l) + 2];
    const double uf = ux * fx + uy * fy + uz * fz;
    const double mx = s * (fx - ux * uf), my = s * (fy - uy * uf), mz = s * (fz - uz * uf);  // MM share
    atomicAdd(&F[3 * j], mx);
    atomicAdd(&F[3 * j + 1], my);
    atomicAdd(&F[3 * j + 2], mz);
    atomicAdd(&F[3 * i], fx - mx);
    atomicAdd(&F[3 * i + 1], fy - my);
    atomicAdd(&F[3 * i + 2], fz - mz);
  }
}

template <class T>
cudaError_t grow_dev(T*& p, size_t& cap, size_t need) {
  if (p && cap >= need) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(&p, (need ? need : 1) * sizeof(T));
  if (e == cudaSuccess) cap = need;
  return e;
}

}  // namespace
}  // namespace nnp

using namespace nnp;

#define MCK(call)                                            \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call); \
  } while (0)

static const char* bad_reason(int bad) {
  if (bad & kBadRange) return "an index is out of range";
  if (bad & kBadRepeat) return "a group index is repeated";
  if (bad & kBadLinkMl) return "a link's ML atom is not in the group";
  if (bad & kBadLinkMm) return "a link's MM atom is in the group";
  if (bad & kBadDist) return "a link distance is not positive";
  return "a link bond has zero length";
}

extern "C" int nnp_eval_mlmm(nnp_ctx* ctx, int64_t n_total, const double* pos, const int32_t* Z,
                             const double* box, int64_t n_ml, const int64_t* ml_index, int32_t n_link,
                             const int64_t* link_ml, const int64_t* link_mm, const double* link_d,
                             int32_t link_Z, double* energy, double* forces) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (n_total <= 0 || !pos || !Z || n_ml <= 0 || !ml_index || n_link < 0 || (n_link > 0 && (!link_ml || !link_mm)))
    return ctx->fail(NNP_ERR_INVALID_ARG, "null argument or empty ML group");
  if (n_ml > n_total) return ctx->fail(NNP_ERR_INVALID_ARG, "more ML atoms than atoms");
  const int lz = link_Z > 0 ? link_Z : 1;
  cudaStream_t st = ctx->stream;
  const bool dev_pos = nnp_ctx::is_device(pos), dev_Z = nnp_ctx::is_device(Z);
  const bool dev_F = forces && nnp_ctx::is_device(forces), dev_E = energy && nnp_ctx::is_device(energy);
  const bool dev_idx = nnp_ctx::is_device(ml_index);
  if (n_link && (nnp_ctx::is_device(link_ml) != dev_idx || nnp_ctx::is_device(link_mm) != dev_idx))
    return ctx->fail(NNP_ERR_INVALID_ARG, "index arrays must all be host or all be device pointers");
  const bool dev_ld = link_d && nnp_ctx::is_device(link_d);
  double3 L = make_double3(0.0, 0.0, 0.0);
  if (box) {
    double b[9];
    if (nnp_ctx::is_device(box)) MCK(cudaMemcpy(b, box, sizeof b, cudaMemcpyDeviceToHost));
    else memcpy(b, box, sizeof b);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        if (r != c && b[3 * r + c] != 0.0) return ctx->fail(NNP_ERR_UNSUPPORTED, "only orthorhombic boxes");
    L = make_double3(b[0], b[4], b[8]);
  }
  const long long n_sub = n_ml + n_link;
  auto& m = ctx->mm;
  MCK(grow_dev(m.pos, m.c_pos, (size_t)3 * n_total));
  MCK(grow_dev(m.Z, m.c_Z, (size_t)n_total));
  MCK(grow_dev(m.F, m.c_F, (size_t)3 * n_total));
  MCK(grow_dev(m.sub_pos, m.c_sub_pos, (size_t)3 * n_sub));
  MCK(grow_dev(m.sub_Z, m.c_sub_Z, (size_t)n_sub));
  MCK(grow_dev(m.sub_F, m.c_sub_F, (size_t)3 * n_sub));
  MCK(grow_dev(m.idx, m.c_idx, (size_t)(n_ml + 2 * n_link)));
  MCK(grow_dev(m.ld, m.c_ld, (size_t)(n_link > 0 ? n_link : 1)));
  MCK(grow_dev(m.E, m.c_E, (size_t)2));
  if (!m.h_bad) MCK(cudaMallocHost(&m.h_bad, sizeof(int)));
  int* d_bad = reinterpret_cast<int*>(m.E + 1);
  MCK(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  const int threads = 256;
  const int64_t *d_ml = ml_index, *d_lml = link_ml, *d_lmm = link_mm;
  const double* d_ld = dev_ld ? link_d : m.ld;
  if (!dev_ld) {  // host distances (or 1 A each) to the device
    m.ld_host.assign((size_t)(n_link > 0 ? n_link : 1), 1.0);
    if (link_d) memcpy(m.ld_host.data(), link_d, sizeof(double) * n_link);
    if (n_link) MCK(cudaMemcpyAsync(m.ld, m.ld_host.data(), sizeof(double) * n_link, cudaMemcpyHostToDevice, st));
  }
  if (!dev_idx) {
    // host index sets: checked here, then copied to the device
    m.mark_host.assign((size_t)n_total, 0);
    for (int64_t k = 0; k < n_ml; ++k) {
      const int64_t a = ml_index[k];
      if (a < 0 || a >= n_total) return ctx->fail(NNP_ERR_INVALID_ARG, "ML index %lld out of range", (long long)a);
      if (m.mark_host[(size_t)a]) return ctx->fail(NNP_ERR_INVALID_ARG, "ML index %lld repeated", (long long)a);
      m.mark_host[(size_t)a] = 1;
    }
    for (int l = 0; l < n_link; ++l) {
      const int64_t i = link_ml[l], j = link_mm[l];
      if (i < 0 || i >= n_total || j < 0 || j >= n_total)
        return ctx->fail(NNP_ERR_INVALID_ARG, "link %d: atom index out of range", l);
      if (!m.mark_host[(size_t)i])
        return ctx->fail(NNP_ERR_INVALID_ARG, "link %d: atom %lld is not in the ML group", l, (long long)i);
      if (m.mark_host[(size_t)j])
        return ctx->fail(NNP_ERR_INVALID_ARG, "link %d: MM atom %lld is in the ML group", l, (long long)j);
    }
    if (dev_ld && n_link) {  // device distances with host indices: checked here too
      m.ld_host.resize((size_t)n_link);
      MCK(cudaMemcpy(m.ld_host.data(), link_d, sizeof(double) * n_link, cudaMemcpyDeviceToHost));
    }
    for (int l = 0; l < n_link; ++l)
      if (!(m.ld_host[(size_t)l] > 0.0)) return ctx->fail(NNP_ERR_INVALID_ARG, "link %d: distance must be positive", l);
    int64_t* h2d = m.idx;
    MCK(cudaMemcpyAsync(h2d, ml_index, sizeof(int64_t) * n_ml, cudaMemcpyHostToDevice, st));
    if (n_link) {
      MCK(cudaMemcpyAsync(h2d + n_ml, link_ml, sizeof(int64_t) * n_link, cudaMemcpyHostToDevice, st));
      MCK(cudaMemcpyAsync(h2d + n_ml + n_link, link_mm, sizeof(int64_t) * n_link, cudaMemcpyHostToDevice, st));
    }
    d_ml = h2d;
    d_lml = h2d + n_ml;
    d_lmm = h2d + n_ml + n_link;
  } else {
    // device index sets: checked by kernels, reported with the evaluation
    MCK(grow_dev(m.mark, m.c_mark, (size_t)n_total));
    MCK(cudaMemsetAsync(m.mark, 0, sizeof(int) * n_total, st));
    const int g = (int)std::min<long long>((n_ml + threads - 1) / threads, (long long)ctx->num_sms * 8);
    k_mlmm_mark<<<g, threads, 0, st>>>(d_ml, n_ml, n_total, m.mark, d_bad);
    if (n_link) k_mlmm_check_links<<<(n_link + threads - 1) / threads, threads, 0, st>>>(d_lml, d_lmm, d_ld, n_link,
                                                                                      n_total, m.mark, d_bad);
  }
  const double* d_pos = pos;
  const int32_t* d_Z = Z;
  if (!dev_pos) {
    MCK(cudaMemcpyAsync(m.pos, pos, sizeof(double) * 3 * n_total, cudaMemcpyHostToDevice, st));
    d_pos = m.pos;
  }
  if (!dev_Z) {
    MCK(cudaMemcpyAsync(m.Z, Z, sizeof(int32_t) * n_total, cudaMemcpyHostToDevice, st));
    d_Z = m.Z;
  }
  const int g_sub = (int)std::min<long long>((n_sub + threads - 1) / threads, (long long)ctx->num_sms * 8);
  k_mlmm_gather<<<g_sub, threads, 0, st>>>(d_pos, d_Z, d_ml, n_ml, n_total, d_lml, d_lmm, d_ld, n_link, lz, L,
                                          m.sub_pos, m.sub_Z, d_bad);
  MCK(cudaGetLastError());
  *m.h_bad = 0;
  MCK(cudaMemcpyAsync(m.h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  // an open system is set up from host positions, copied outside this stream
  if (!box) MCK(cudaStreamSynchronize(st));
  // the NNP on the subsystem (one system, the caller's box); it synchronises the stream
  const int64_t off[2] = {0, n_sub};
  int rc = ctx->evaluate(1, off, m.sub_pos, m.sub_Z, box, m.E, m.sub_F, true);
  if (rc) cudaStreamSynchronize(st);  // the flag copy has landed
  if (*m.h_bad) return ctx->fail(NNP_ERR_INVALID_ARG, "ML/MM input rejected: %s", bad_reason(*m.h_bad));
  if (rc) return rc;
  double* d_F = dev_F ? forces : m.F;
  MCK(cudaMemsetAsync(d_F, 0, sizeof(double) * 3 * n_total, st));
  const int g_ml = (int)std::min<long long>((n_ml + threads - 1) / threads, (long long)ctx->num_sms * 8);
  k_mlmm_scatter_ml<<<g_ml, threads, 0, st>>>(m.sub_F, d_ml, n_ml, d_F);
  if (n_link)
    k_mlmm_links<<<(n_link + threads - 1) / threads, threads, 0, st>>>(d_pos, m.sub_F, n_ml, d_lml, d_lmm, d_ld, n_link,
                                                                       L, d_F);
  MCK(cudaGetLastError());
  if (energy) MCK(cudaMemcpyAsync(energy, m.E, sizeof(double), dev_E ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (forces && !dev_F)
    MCK(cudaMemcpyAsync(forces, m.F, sizeof(double) * 3 * n_total, cudaMemcpyDeviceToHost, st));
  MCK(cudaStreamSynchronize(st));
  return NNP_OK;
}
