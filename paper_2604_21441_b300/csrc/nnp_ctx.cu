// nnp_ctx.cu -- context life cycle, weight upload and the stage profiler.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nnp_host.h"

using namespace nnp;

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

int nnp_ctx::init_device() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  if (cfg.stream) {
    stream = (cudaStream_t)cfg.stream;
    own_stream = false;
  } else {
    CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    own_stream = true;
  }
  if (cfg.flags & NNP_FLAG_STAGE_EVENTS)
    for (auto& ev : stage_ev) CK(cudaEventCreate(&ev));
  CK(neighbors_set_smem_limits());
  CK(aev_set_smem_limits());
  CK(mlp_f32_set_smem_limits());
  CK(cudaMalloc(&b_seg, sizeof(int) * (kMaxS + 2)));
  CK(cudaMalloc(&b_flags, sizeof(int) * kNumFlags));
  CK(cudaMemset(b_flags, 0, sizeof(int) * kNumFlags));
  CK(cudaMalloc(&d_io, sizeof(EvalIO)));
  CK(cudaMallocHost(&h_io, sizeof(EvalIO)));
  CK(cudaMallocHost(&h_flags, sizeof(int) * kNumFlags));
  memset(h_flags, 0, sizeof(int) * kNumFlags);
  signed char lut[128];
  for (int z = 0; z < 128; ++z) lut[z] = -1;
  for (int s = 0; s < P.S; ++s) lut[cfg.atomic_numbers[s]] = (signed char)s;
  CK(cudaMalloc(&d_zlut, 128));
  CK(cudaMemcpy(d_zlut, lut, 128, cudaMemcpyHostToDevice));
  // weights: W1 (D x 160), W2, W3, W4, b1..b4, W1T, W2T, W3T per species
  const size_t D = P.D;
  wf32_stride = D * kH1 + kH1 * kH2 + kH2 * kH3 + kH3 + kH1 + kH2 + kH3 + 1 + kH1 * D + kH2 * kH1 +
                kH3 * kH2;
  wf32_stride = (wf32_stride + 63) / 64 * 64;
  CK(cudaMalloc(&b_wf32, sizeof(float) * wf32_stride * P.S));
  CK(cudaMemset(b_wf32, 0, sizeof(float) * wf32_stride * P.S));
  for (int s = 0; s < P.S; ++s) {
    float* p = b_wf32 + wf32_stride * s;
    wf32.W[s][0] = p; p += D * kH1;
    wf32.W[s][1] = p; p += kH1 * kH2;
    wf32.W[s][2] = p; p += kH2 * kH3;
    wf32.W[s][3] = p; p += kH3;
    wf32.b[s][0] = p; p += kH1;
    wf32.b[s][1] = p; p += kH2;
    wf32.b[s][2] = p; p += kH3;
    wf32.b[s][3] = p; p += 1;
    wf32.WT[s][0] = p; p += kH1 * D;
    wf32.WT[s][1] = p; p += kH2 * kH1;
    wf32.WT[s][2] = p; p += kH3 * kH2;
  }
  host_weights.assign((size_t)nnp_param_count(this), 0.f);
  if (cfg.precision != NNP_FP32) {
    int rc = mlp_tc_init(this);
    if (rc) return rc;
  }
  long long n0 = cfg.max_atoms > 0 ? cfg.max_atoms : 4096;
  int B0 = cfg.max_systems > 0 ? cfg.max_systems : 1;
  long long cells0 = std::max<long long>(64, 2 * n0);
  int rc = ensure_capacity(n0, B0, cells0 * P.S, n0 + kTileRows * P.S);
  if (rc) return rc;
  CK(cudaStreamSynchronize(stream));
  return NNP_OK;
}

nnp_ctx::~nnp_ctx() {
  if (stream) cudaStreamSynchronize(stream);
  invalidate_graph();
  mlp_tc_free(this);
  void* bufs[] = {b_bin_count, b_bin_start, b_bin_len, b_atom_bin, b_atom_slot, b_atom_cell,
                  b_atom_sys, b_atom_off, b_row_atom, b_row_info, b_row_cell, b_pos4, b_cnt_r,
                  b_cnt_a, b_nbr_r, b_G, b_dEdG, b_Ei, b_Gh, b_sys, b_pos_stage,
                  b_Z_stage, b_F_stage, b_E_stage, b_seg, b_flags, d_zlut, d_io, b_wf32};
  for (void* p : bufs)
    if (p) cudaFree(p);
  for (auto& ev : stage_ev)
    if (ev) cudaEventDestroy(ev);
  if (h_io) cudaFreeHost(h_io);
  if (h_flags) cudaFreeHost(h_flags);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

static bool dev_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int nnp_ctx::set_weights(int s, const float* const W[4], const float* const b[4]) {
  const int D = P.D;
  const int fin[4] = {D, kH1, kH2, kH3}, fout[4] = {kH1, kH2, kH3, 1};
  std::vector<float> w[4], bb[4];
  for (int l = 0; l < 4; ++l) {
    w[l].resize((size_t)fin[l] * fout[l]);
    bb[l].resize(fout[l]);
    const size_t wb = sizeof(float) * w[l].size(), bbytes = sizeof(float) * bb[l].size();
    if (dev_ptr(W[l])) CK(cudaMemcpy(w[l].data(), W[l], wb, cudaMemcpyDeviceToHost));
    else memcpy(w[l].data(), W[l], wb);
    if (dev_ptr(b[l])) CK(cudaMemcpy(bb[l].data(), b[l], bbytes, cudaMemcpyDeviceToHost));
    else memcpy(bb[l].data(), b[l], bbytes);
    for (float x : w[l])
      if (!std::isfinite(x)) return fail(NNP_ERR_INVALID_ARG, "non-finite weight in layer %d", l);
    for (float x : bb[l])
      if (!std::isfinite(x)) return fail(NNP_ERR_INVALID_ARG, "non-finite bias in layer %d", l);
  }
  std::vector<float> blob(wf32_stride, 0.f);
  float* p = blob.data();
  auto put = [&](const std::vector<float>& v) { memcpy(p, v.data(), sizeof(float) * v.size()); p += v.size(); };
  put(w[0]); put(w[1]); put(w[2]); put(w[3]);
  put(bb[0]); put(bb[1]); put(bb[2]); put(bb[3]);
  for (int l = 0; l < 3; ++l) {  // transposed copies (fan_out x fan_in)
    for (int o = 0; o < fout[l]; ++o)
      for (int i = 0; i < fin[l]; ++i) p[(size_t)o * fin[l] + i] = w[l][(size_t)i * fout[l] + o];
    p += (size_t)fin[l] * fout[l];
  }
  CK(cudaStreamSynchronize(stream));
  CK(cudaMemcpy(b_wf32 + wf32_stride * s, blob.data(), sizeof(float) * wf32_stride,
                cudaMemcpyHostToDevice));
  // packed FP32 copy in the nnp_param_count layout: W1 b1 W2 b2 W3 b3 W4 b4
  size_t per = 0;
  for (int l = 0; l < 4; ++l) per += (size_t)fin[l] * fout[l] + fout[l];
  float* hp = host_weights.data() + per * s;
  for (int l = 0; l < 4; ++l) {
    memcpy(hp, w[l].data(), sizeof(float) * w[l].size()); hp += w[l].size();
    memcpy(hp, bb[l].data(), sizeof(float) * bb[l].size()); hp += bb[l].size();
  }
  if (cfg.precision != NNP_FP32) {
    int rc = mlp_tc_set_weights(this, s, host_weights.data() + per * s);
    if (rc) return rc;
  }
  has_weights[s] = true;
  return NNP_OK;
}

int nnp_ctx::force_match_grad(const double*, const double*, double*, double*) {
  return fail(NNP_ERR_UNSUPPORTED, "force-matching gradients are not built yet");
}

int nnp_ctx::profile_stages(double* out, int n_out) {
  if (!stage_ev[0]) return fail(NNP_ERR_UNSUPPORTED, "context was created without NNP_FLAG_STAGE_EVENTS");
  if (!has_state) return fail(NNP_ERR_NO_STATE, "no evaluation to profile");
  CK(cudaEventSynchronize(stage_ev[5]));
  for (int k = 0; k < 5 && k < n_out; ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, stage_ev[k], stage_ev[k + 1]));
    out[k] = ms;
  }
  return NNP_OK;
}
