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
  CK(cudaMalloc(&b_queue, sizeof(int) * kQueueWords));
  CK(cudaMemset(b_queue, 0, sizeof(int) * kQueueWords));
  CK(cudaMalloc(&d_io, sizeof(EvalIO)));
  for (auto& sg : stages) {
    CK(cudaMallocHost(&sg.io, sizeof(EvalIO)));
    memset(sg.io, 0, sizeof(EvalIO));
    CK(cudaEventCreateWithFlags(&sg.ev, cudaEventDisableTiming));
  }
  h_io = stages[0].io;
  CK(cudaMallocHost(&h_flags, sizeof(int) * kNumFlags));
  memset(h_flags, 0, sizeof(int) * kNumFlags);
  signed char lut[128];
  for (int z = 0; z < 128; ++z) lut[z] = -1;
  for (int s = 0; s < P.S; ++s) lut[cfg.atomic_numbers[s]] = (signed char)s;
  CK(cudaMalloc(&d_zlut, 128));
  CK(cudaMemcpy(d_zlut, lut, 128, cudaMemcpyHostToDevice));
  // weights: W1 (D x 160), W2, W3, W4, b1..b4, W1T, W2T, W3T per species; b4
  // takes four floats so that every array starts on 16 bytes (float4 loads)
  const size_t D = P.D;
  wf32_stride = D * kH1 + kH1 * kH2 + kH2 * kH3 + kH3 + kH1 + kH2 + kH3 + 4 + kH1 * D + kH2 * kH1 +
                kH3 * kH2;
  wf32_stride = (wf32_stride + 63) / 64 * 64;
  // one table per ensemble member (member m, species s at (m S + s) strides),
  // then the charge network's (set n_members) with NNP_FLAG_CHARGES
  const int sets = n_members + (has_charges ? 1 : 0);
  const size_t tables = (size_t)sets * P.S;
  CK(cudaMalloc(&b_wf32, sizeof(float) * wf32_stride * tables));
  CK(cudaMemset(b_wf32, 0, sizeof(float) * wf32_stride * tables));
  wf32m.assign((size_t)sets, MlpF32Weights{});
  for (int m = 0; m < sets; ++m)
    for (int s = 0; s < P.S; ++s) {
      MlpF32Weights& t = wf32m[(size_t)m];
      float* p = b_wf32 + wf32_stride * ((size_t)m * P.S + s);
      t.W[s][0] = p; p += D * kH1;
      t.W[s][1] = p; p += kH1 * kH2;
      t.W[s][2] = p; p += kH2 * kH3;
      t.W[s][3] = p; p += kH3;
      t.b[s][0] = p; p += kH1;
      t.b[s][1] = p; p += kH2;
      t.b[s][2] = p; p += kH3;
      t.b[s][3] = p; p += 4;
      t.WT[s][0] = p; p += kH1 * D;
      t.WT[s][1] = p; p += kH2 * kH1;
      t.WT[s][2] = p; p += kH3 * kH2;
    }
  wf32 = wf32m[0];
  has_w.assign((size_t)sets * kMaxS, 0);
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
                  b_cnt_a, b_nbr_r, b_G, b_dEdG, b_Ei, b_Gh, b_g1, b_sys, b_pos_stage,
                  b_Z_stage, b_F_stage, b_E_stage, b_seg, b_flags, b_queue, d_zlut, d_io, b_wf32,
                  fm_z, fm_dz, fm_t, fm_p, fm_v, fm_ref, fm_grad, fm_jobs,
                  mm.pos, mm.F, mm.sub_pos, mm.sub_F, mm.ld, mm.E, mm.Z, mm.sub_Z, mm.idx, mm.mark,
                  b_pair_cur, b_pairs_stage, b_shifts_stage, d_ee, d_io_q, b_ee_mmhi, b_ee_mmlo,
                  b_ee_mlhi, b_ee_mllo, b_ee_V, b_ee_field, b_ee_qatom, b_ee_qout, b_ee_mmF, b_ee_mmpos,
                  b_ee_mmq, b_ee_sums, b_ee_qrows, b_ee_dqdG};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (mm.h_bad) cudaFreeHost(mm.h_bad);
  if (h_ee) cudaFreeHost(h_ee);
  for (auto& ev : stage_ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : fm_ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& sg : stages) {
    if (sg.io) cudaFreeHost(sg.io);
    if (sg.sys) cudaFreeHost(sg.sys);
    if (sg.ev) cudaEventDestroy(sg.ev);
  }
  if (h_flags) cudaFreeHost(h_flags);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

bool nnp_ctx::is_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Member m's weights.  With an ensemble of M members, the output layer (W4,
// b4) is stored divided by M, so that the networks' sum over members is
// their mean: energies and dE/dG add up member by member.
int nnp_ctx::set_weights(int m, int s, const float* const W[4], const float* const b[4]) {
  const int D = P.D;
  const int fin[4] = {D, kH1, kH2, kH3}, fout[4] = {kH1, kH2, kH3, 1};
  std::vector<float> w[4], bb[4];
  for (int l = 0; l < 4; ++l) {
    w[l].resize((size_t)fin[l] * fout[l]);
    bb[l].resize(fout[l]);
    const size_t wb = sizeof(float) * w[l].size(), bbytes = sizeof(float) * bb[l].size();
    if (is_device(W[l])) CK(cudaMemcpy(w[l].data(), W[l], wb, cudaMemcpyDeviceToHost));
    else memcpy(w[l].data(), W[l], wb);
    if (is_device(b[l])) CK(cudaMemcpy(bb[l].data(), b[l], bbytes, cudaMemcpyDeviceToHost));
    else memcpy(bb[l].data(), b[l], bbytes);
    for (float x : w[l])
      if (!std::isfinite(x)) return fail(NNP_ERR_INVALID_ARG, "non-finite weight in layer %d", l);
    for (float x : bb[l])
      if (!std::isfinite(x)) return fail(NNP_ERR_INVALID_ARG, "non-finite bias in layer %d", l);
  }
  std::vector<float> blob(wf32_stride, 0.f);
  float* p = blob.data();
  auto put = [&](const std::vector<float>& v) { memcpy(p, v.data(), sizeof(float) * v.size()); p += v.size(); };
  std::vector<float> w4 = w[3], b4 = bb[3];
  if (m < n_members) {  // ensemble members: the mean (the charge network is not averaged)
    for (float& x : w4) x /= (float)n_members;
    for (float& x : b4) x /= (float)n_members;
  }
  put(w[0]); put(w[1]); put(w[2]); put(w4);
  put(bb[0]); put(bb[1]); put(bb[2]); put(b4);
  p += 3;  // b4 padded to four floats
  for (int l = 0; l < 3; ++l) {  // transposed copies (fan_out x fan_in)
    for (int o = 0; o < fout[l]; ++o)
      for (int i = 0; i < fin[l]; ++i) p[(size_t)o * fin[l] + i] = w[l][(size_t)i * fout[l] + o];
    p += (size_t)fin[l] * fout[l];
  }
  CK(cudaStreamSynchronize(stream));
  CK(cudaMemcpy(b_wf32 + wf32_stride * ((size_t)m * P.S + s), blob.data(), sizeof(float) * wf32_stride,
                cudaMemcpyHostToDevice));
  // packed FP32 copy in the nnp_param_count layout: W1 b1 W2 b2 W3 b3 W4 b4
  // (member 0 keeps it for force matching and FP8 re-quantisation)
  size_t per = 0;
  for (int l = 0; l < 4; ++l) per += (size_t)fin[l] * fout[l] + fout[l];
  std::vector<float> packed(per);
  float* hp = packed.data();
  for (int l = 0; l < 4; ++l) {
    memcpy(hp, w[l].data(), sizeof(float) * w[l].size()); hp += w[l].size();
    memcpy(hp, bb[l].data(), sizeof(float) * bb[l].size()); hp += bb[l].size();
  }
  if (m == 0) memcpy(host_weights.data() + per * s, packed.data(), sizeof(float) * per);
  if (cfg.precision != NNP_FP32) {
    int rc = mlp_tc_set_weights(this, m, s, packed.data());
    if (rc) return rc;
  }
  has_w[(size_t)m * kMaxS + s] = 1;
  return NNP_OK;
}

// v = 2 (F - Fref) / (3n) and loss = |F - Fref|^2 / (3n) (FP64).
__global__ void k_fm_v(const double* __restrict__ F, const double* __restrict__ Fref, long long n3,
                       double scale, double* v, double* loss) {
  double part = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n3;
       q += (long long)gridDim.x * blockDim.x) {
    const double e = F[q] - Fref[q];
    v[q] = 2.0 * e * scale;
    part += e * e;
  }
  for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part * scale);
}

template <class T>
static cudaError_t grow_buf(T*& p, size_t& cap, size_t need) {
  if (p && cap >= need) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(&p, need * sizeof(T));
  if (e == cudaSuccess) cap = need;
  return e;
}

// Force matching (Eq. 2's forces as a training signal).  For an ensemble
// of M members, E = sum_m E_m with each member's output layer stored divided
// by M, so dL/dtheta_m is the single-network formula applied to member m's
// stored network (its output weights' gradient scaled by 1/M, the ratio of
// stored to given weights); the loss's v = dL/dF comes from the ensemble's F.
int nnp_ctx::force_match_grad(const double* v, const double* Fref, double* loss, double* grad) {
  if (!has_state) return fail(NNP_ERR_NO_STATE, "nnp_force_match_grad needs a previous nnp_eval");
  if (!grad) return fail(NNP_ERR_INVALID_ARG, "null gradient output");
  if (!v && !Fref) return fail(NNP_ERR_INVALID_ARG, "pass v = dL/dF or the reference forces");
  const long long n = last_n, rows = last_rows;
  const int D = P.D;
  const size_t npar = (size_t)nnp_param_count(this);
  const size_t per_member = npar / (size_t)n_members;
  const bool prof = stage_ev[0] != nullptr;
  if (prof && !fm_ev[0])
    for (auto& ev : fm_ev) CK(cudaEventCreate(&ev));
  CK(cudaStreamSynchronize(stream));  // the staging slot below is rewritten
  // species segments of the last evaluation (rows per species), for the
  // weight-gradient jobs; the stream is idle, so this copy waits for nothing
  int seg[kMaxS + 2];
  CK(cudaMemcpy(seg, b_seg, sizeof(seg), cudaMemcpyDeviceToHost));
  CK(grow_buf(fm_z, fm_cap, (size_t)rows * 384));
  CK(grow_buf(fm_dz, fm_cap2, (size_t)rows * 384));
  CK(grow_buf(fm_t, fm_cap3, (size_t)rows * 384));
  CK(grow_buf(fm_p, fm_cap4, (size_t)rows * 384));
  CK(grow_buf(fm_v, fm_vcap, (size_t)n * 3));
  CK(grow_buf(fm_ref, fm_refcap, (size_t)n * 3));
  CK(grow_buf(fm_grad, fm_gcap, npar + 1));  // last entry: loss
  const Workspace w = workspace();
  if (prof) CK(cudaEventRecord(fm_ev[0], stream));
  // 1. FP32 forces of the last evaluated configuration into internal buffers
  EvalIO io = *h_io;
  io.forces = b_F_stage;
  io.energies = b_E_stage;
  *h_io = io;
  CK(cudaMemcpyAsync(d_io, h_io, sizeof(EvalIO), cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(b_F_stage, 0, sizeof(double) * 3 * n, stream));
  CK(cudaMemsetAsync(b_E_stage, 0, sizeof(double) * last_B, stream));
  launch_aev_fwd(rows, num_sms, stream, b_sys, P, w, 0);
  const int g_tiles = (int)std::max<long long>(1, std::min<long long>(rows / 64, (long long)num_sms));
  for (int m = 0; m < n_members; ++m)  // members add up their E_i and dE/dG
    launch_mlp_f32(g_tiles, stream, d_io, P, w, wf32m[(size_t)m], m > 0 ? 1 : 0);
  launch_aev_bwd(rows, num_sms, stream, d_io, b_sys, P, w);
  if (prof) CK(cudaEventRecord(fm_ev[1], stream));
  // 2. v = dL/dF (given, or from the reference forces)
  double* lossd = fm_grad + npar;
  CK(cudaMemsetAsync(fm_grad, 0, sizeof(double) * (npar + 1), stream));
  if (Fref) {
    const double* fr = Fref;
    if (!is_device(Fref)) {
      CK(cudaMemcpyAsync(fm_ref, Fref, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, stream));
      fr = fm_ref;
    }
    k_fm_v<<<std::max(1, std::min(num_sms * 4, (int)((3 * n + 255) / 256))), 256, 0, stream>>>(
        b_F_stage, fr, 3 * n, 1.0 / (3.0 * (double)n), fm_v, lossd);
  } else {
    CK(cudaMemcpyAsync(fm_v, v, sizeof(double) * 3 * n,
                       is_device(v) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream));
  }
  // 3. tangent descriptors dG = J_G v (into the dE/dG buffer)
  launch_aev_jvp(rows, num_sms, stream, b_sys, P, w, fm_v, b_dEdG);
  if (prof) CK(cudaEventRecord(fm_ev[2], stream));
  // weight-gradient jobs per member, species, layer, 64 x 64 tile and
  // 256-row segment (the segment bounds are the last evaluation's); the
  // device list is kept while the segments stay the same
  std::vector<FmJob>& jobs = fm_job_list;
  const int fin[4] = {D, kH1, kH2, kH3}, fout[4] = {kH1, kH2, kH3, 1};
  const size_t per = per_member / P.S;
  const bool same_jobs = !jobs.empty() && std::equal(seg, seg + P.S + 1, fm_job_seg);
  if (!same_jobs) jobs.clear();
  for (int m = 0; m < n_members && !same_jobs; ++m)
    for (int sp = 0; sp < P.S; ++sp) {
      size_t off = per_member * m + per * sp;
      size_t woff[4], boff[4];
      for (int l = 0; l < 4; ++l) {
        woff[l] = off;
        off += (size_t)fin[l] * fout[l];
        boff[l] = off;
        off += fout[l];
      }
      for (int r0 = seg[sp]; r0 < seg[sp + 1]; r0 += 256) {
        const int r1 = std::min(seg[sp + 1], r0 + 256);
        for (int l = 0; l < 4; ++l)
          for (int i0 = 0; i0 < fin[l]; i0 += 64)
            for (int o0 = 0; o0 < fout[l]; o0 += 64)
              jobs.push_back(FmJob{l + 1, i0, o0, r0, r1, l == 3 ? 1.0f / (float)n_members : 1.0f,
                                   (long long)woff[l], (long long)boff[l]});
      }
    }
  if (!same_jobs) {
    CK(grow_buf(fm_jobs, fm_jcap, jobs.size() + 1));
    CK(cudaMemcpyAsync(fm_jobs, jobs.data(), sizeof(FmJob) * jobs.size(), cudaMemcpyHostToDevice, stream));
    std::copy(seg, seg + P.S + 1, fm_job_seg);
  }
  const int jobs_per_member = (int)jobs.size() / n_members;
  for (int m = 0; m < n_members; ++m) {
    // 4. member m's network: primal + tangent forward, reverse adjoints
    launch_fm(g_tiles, stream, P, w, wf32m[(size_t)m], b_dEdG, fm_z, fm_dz, fm_t, fm_p);
    if (prof) CK(cudaEventRecord(fm_ev[3 + 2 * m], stream));
    // 5. its weight-gradient jobs (they read the buffers step 4 wrote)
    launch_fm_wgrad(std::max(1, std::min(jobs_per_member, num_sms * 8)), stream, P,
                    fm_jobs + (size_t)m * jobs_per_member, jobs_per_member, b_G, b_dEdG, fm_z, fm_dz, fm_t,
                    fm_p, fm_grad);
    if (prof) CK(cudaEventRecord(fm_ev[4 + 2 * m], stream));
  }
  CK(cudaGetLastError());
  fm_profiled_members = prof ? n_members : 0;
  // 6. results
  CK(cudaMemcpyAsync(grad, fm_grad, sizeof(double) * npar,
                     is_device(grad) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
  double lh = 0.0;
  if (loss) CK(cudaMemcpyAsync(&lh, lossd, sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  if (loss) *loss = Fref ? lh : 0.0;
  return NNP_OK;
}

// Stage durations of the last nnp_force_match_grad: forces, tangent
// descriptors, networks (all members), weight gradients (all members).
int nnp_ctx::profile_force_match(double* out, int n_out) {
  if (!stage_ev[0]) return fail(NNP_ERR_UNSUPPORTED, "context was created without NNP_FLAG_STAGE_EVENTS");
  if (fm_profiled_members <= 0) return fail(NNP_ERR_NO_STATE, "no force-matching gradient to profile");
  const int M = fm_profiled_members;
  CK(cudaEventSynchronize(fm_ev[2 + 2 * M]));
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, fm_ev[0], fm_ev[1]));
  t[0] = ms;
  CK(cudaEventElapsedTime(&ms, fm_ev[1], fm_ev[2]));
  t[1] = ms;
  for (int m = 0; m < M; ++m) {
    // member m's network starts where the previous member's jobs ended (the
    // first after the tangent descriptors and the host's job list)
    CK(cudaEventElapsedTime(&ms, m == 0 ? fm_ev[2] : fm_ev[2 + 2 * m], fm_ev[3 + 2 * m]));
    t[2] += ms;
    CK(cudaEventElapsedTime(&ms, fm_ev[3 + 2 * m], fm_ev[4 + 2 * m]));
    t[3] += ms;
  }
  for (int k = 0; k < 4 && k < n_out; ++k) out[k] = t[k];
  return NNP_OK;
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
