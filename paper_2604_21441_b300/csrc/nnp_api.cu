// nnp_api.cu -- the C ABI of libnnp (include/nnp.h) and its host-side
// orchestration: argument checks, cell-grid set-up per system, device
// workspaces that grow on demand, the per-evaluation kernel sequence
// (captured once into a CUDA graph and replayed), device flag checks with
// neighbour-list regrowth, and host/device pointer staging.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nnp.h"
#include "nnp_host.h"

using namespace nnp;

namespace {

thread_local std::string g_create_error;

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Page-locked host memory that the device addresses in place (unified
// addressing: cudaHostAlloc'd or registered buffers): its device address,
// else nullptr.
const void* mapped_host_ptr(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int grid_for(long long items, int per_block, int cap) {
  long long g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
// context helpers

int nnp_ctx::fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  err = buf;
  return code;
}

int nnp_ctx::cuda_fail(cudaError_t e, const char* what) {
  return fail(NNP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <class T>
static cudaError_t grow(T*& p, size_t& cap, size_t need) {
  if (need <= cap && p) return cudaSuccess;
  size_t nc = std::max(need, cap + cap / 2);
  if (p) cudaFree(p);
  p = nullptr;
  cudaError_t e = cudaMalloc(&p, nc * sizeof(T));
  if (e != cudaSuccess) { cap = 0; return e; }
  cap = nc;
  return cudaSuccess;
}

int nnp_ctx::ensure_capacity(long long n, int B, long long bins, long long rows) {
  bool changed = false;
  auto G = [&](auto*& p, size_t& cap, size_t need) -> cudaError_t {
    size_t before = cap;
    auto* old = p;
    cudaError_t e = grow(p, cap, need);
    if (cap != before || p != old) changed = true;
    return e;
  };
  cudaError_t e;
#define GR(p, c, need) if ((e = G(p, c, need)) != cudaSuccess) return cuda_fail(e, "cudaMalloc " #p)
  GR(b_bin_count, c_bins, (size_t)bins);
  if (changed) {
    CK(cudaMemsetAsync(b_bin_count, 0, sizeof(int) * c_bins, stream));
  }
  GR(b_bin_start, c_bins1, (size_t)bins + 1);
  GR(b_bin_len, c_bins2, (size_t)bins);
  GR(b_atom_bin, c_atoms1, (size_t)n);
  GR(b_atom_slot, c_atoms2, (size_t)n);
  GR(b_atom_off, c_atoms3, (size_t)n);
  GR(b_atom_cell, c_atoms4, (size_t)n);
  GR(b_atom_sys, c_atoms5, (size_t)n);
  GR(b_row_atom, c_rows1, (size_t)rows);
  GR(b_pos4, c_rows2, (size_t)rows);
  GR(b_row_info, c_rows3, (size_t)rows);
  GR(b_row_cell, c_rows4, (size_t)rows);
  GR(b_cnt_r, c_rows5, (size_t)rows * kMaxS);
  GR(b_cnt_a, c_rows6, (size_t)rows * kMaxS);
  GR(b_nbr_r, c_nbr_r, (size_t)rows * cap_r);
  GR(b_G, c_G, (size_t)rows * P.D);
  __nv_bfloat16* gh_old = b_Gh;
  GR(b_Gh, c_Gh, (size_t)rows * ((P.D + 63) / 64 * 64));  // swizzled BF16 tiles (or E4M3 ones)
  // E4M3 tiles: the columns past D up to the next 32 are read by the last MMA
  // of layer 1 and never written, so they must hold zeros
  if (b_Gh != gh_old) CK(cudaMemsetAsync(b_Gh, 0, sizeof(__nv_bfloat16) * c_Gh, stream));
  GR(b_dEdG, c_dEdG, (size_t)rows * P.D);
  GR(b_Ei, c_Ei, (size_t)rows);
  if (ens_wide()) GR(b_g1, c_g1, (size_t)((rows + 127) / 128) * n_members * kG1TileBytes);
  GR(b_sys, c_sys, (size_t)B);
  GR(b_pos_stage, c_pos_stage, (size_t)n * 3);
  GR(b_Z_stage, c_Z_stage, (size_t)n);
  GR(b_F_stage, c_F_stage, (size_t)n * 3);
  GR(b_E_stage, c_E_stage, (size_t)B);
  if (ext_mode) GR(b_pair_cur, c_pair_cur, (size_t)rows * 2 * kMaxS);
#undef GR
  if (changed) invalidate_graph();
  return NNP_OK;
}

Workspace nnp_ctx::workspace() const {
  Workspace w{};
  w.bin_count = b_bin_count;
  w.bin_start = b_bin_start;
  w.bin_len = b_bin_len;
  w.atom_bin = b_atom_bin;
  w.atom_slot = b_atom_slot;
  w.atom_off = b_atom_off;
  w.atom_cell = b_atom_cell;
  w.atom_sys = b_atom_sys;
  w.seg = b_seg;
  w.row_atom = b_row_atom;
  w.pos4 = b_pos4;
  w.row_info = b_row_info;
  w.row_cell = b_row_cell;
  w.cnt_r = b_cnt_r;
  w.cnt_a = b_cnt_a;
  w.nbr_r = b_nbr_r;
  w.G = b_G;
  w.Gh = b_Gh;
  w.dEdG = b_dEdG;
  w.Ei = b_Ei;
  w.flags = b_flags;
  w.queue = b_queue;
  w.q8 = b_q8;
  w.cap_r = cap_r;
  w.cap_a = cap_a;
  w.max_rows = (long long)c_rows1;
  return w;
}

void nnp_ctx::invalidate_graph() {
  if (gexec) cudaGraphExecDestroy(gexec);
  gexec = nullptr;
  g_key_n = -1;
}

// The kernel sequence of one evaluation (stream-ordered; capturable).
int nnp_ctx::launch_pipeline(long long n, int B, long long bins, long long rows, bool calib) {
  const Workspace w = workspace();
  const int nsm = num_sms;
  const int g_atoms = grid_for(n, 256, nsm * 8);
  const int g_cells = grid_for(total_cells * ((tune.nbr_dyn & 2) ? 2 : 1), kNbrThreads / 32, nsm * tune.nbr);
  const int g_bins = grid_for(bins * 32, 256, nsm * 16);
  const EvalIO* io = d_io;
  const SysDesc* sys = b_sys;
  int launches = 0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(stream, &cs));
  const bool capturing = cs == cudaStreamCaptureStatusActive;
  mark_stage(0, capturing);
  const int sort = (cfg.flags & NNP_FLAG_NONDETERMINISTIC_BINS) ? 0 : 1;
  if (rows <= kCellsRowsSmall) {  // small systems: the four binning steps in one block
    k_cells_small<<<1, 1024, sizeof(int) * kScanSmemBinsSmall, stream>>>(io, sys, d_zlut, P.S, sort, w); ++launches;
  } else {
    k_bin<<<g_atoms, 256, 0, stream>>>(io, sys, d_zlut, w); ++launches;
    k_scan<<<1, 1024, sizeof(int) * kScanSmemBins, stream>>>(io, P.S, w); ++launches;
    k_scatter<<<g_atoms, 256, 0, stream>>>(io, w); ++launches;
    k_binsort<<<g_bins, 256, 0, stream>>>(io, P.S, sort, w); ++launches;
  }
  mark_stage(1, capturing);
  if (ext_mode) {  // the caller's pair list instead of the cell search
    const int g_rows = grid_for(rows, 256, nsm * 8), g_pairs = nsm * 16;
    k_pairs_prep<<<g_rows, 256, 0, stream>>>(P.S, w);
    k_pairs_count<<<g_pairs, 256, 0, stream>>>(io, sys, P, w);
    k_pairs_offsets<<<g_rows, 256, 0, stream>>>(io, P.S, w, b_pair_cur);
    k_pairs_fill<<<g_pairs, 256, 0, stream>>>(io, sys, P, w, b_pair_cur);
    launches += 4;
  } else {
    launch_neighbors(g_cells, stream, io, sys, P, w, rows, total_cells, nsm, tune.nbr_dyn); ++launches;
  }
  mark_stage(2, capturing);
  if (calib) {  // FP8 calibration: FP32 descriptor, then the activation ranges
    launch_aev_fwd(rows, nsm, stream, sys, P, w, kGFp32, tune.fwd, tune.fwd_tile);
    int rc = launch_fp8_calib(this, stream, rows);
    if (rc) return rc;
    CK(cudaGetLastError());
    return NNP_OK;
  }
  const int gmode = cfg.precision == NNP_FP32 ? kGFp32 : (cfg.precision == NNP_BF16 ? kGBf16 : kGFp8);
  launch_aev_fwd(rows, nsm, stream, sys, P, w, gmode, tune.fwd, tune.fwd_tile); ++launches;
  mark_stage(3, capturing);
  const int g_tiles = (int)std::min<long long>(rows / 64, (long long)nsm);
  if (cfg.precision == NNP_FP32) {
    for (int m = 0; m < n_members; ++m) {  // ensemble members add up (mean by the stored 1/M)
      launch_mlp_f32(std::max(1, g_tiles), stream, io, P, w, wf32m[(size_t)m], m > 0 ? 1 : 0);
      ++launches;
    }
  } else {  // ensemble members side by side in one launch, outputs added with reductions
    if (n_members > 1) {
      CK(cudaMemsetAsync(b_Ei, 0, sizeof(float) * (size_t)rows, stream));
      // wide networks write dE/dG once, from one product over the members
      if (!ens_wide()) CK(cudaMemsetAsync(b_dEdG, 0, sizeof(float) * (size_t)rows * P.D, stream));
    }
    int rc = launch_mlp_tc(this, stream, rows, 0, n_members, n_members > 1 ? 1 : 0);
    if (rc) return rc;
    launches += ens_wide() ? 2 : 1;
  }
  if (ee_mode) {  // embedding: potentials, charge network, dE/dG of the charges
    int rc = launch_ee_pre(rows, w, launches);
    if (rc) return rc;
  }
  mark_stage(4, capturing);
  launch_aev_bwd(rows, nsm, stream, io, sys, P, w, tune.bwd, tune.bwd_tile); ++launches;
  if (ee_mode) launch_ee_post(launches);  // charges, embedding energy, ML and MM forces
  mark_stage(5, capturing);
  CK(cudaGetLastError());
  launches_per_eval = launches;
  return NNP_OK;
}

void nnp_ctx::mark_stage(int k, bool capturing) {
  if (!stage_ev[k]) return;
  if (capturing) cudaEventRecordWithFlags(stage_ev[k], stream, cudaEventRecordExternal);
  else cudaEventRecord(stage_ev[k], stream);
}

// FP8 form: one synchronous pass of the FP32 descriptor and network forward
// over this input sets the activation ranges (Workspace::q8).  Runs before the
// evaluation proper, outside any graph; the device flags accumulated by
// earlier asynchronous evaluations are kept for nnp_sync.  Species absent
// from this input stay uncalibrated; a later input that has one makes the
// network kernel raise kFlagFp8Uncal, and that evaluation is calibrated again
// (the ranges only grow) and redone.  An input without the absent species
// needs no new pass.  Returns -1 if the lists were regrown.
int nnp_ctx::calibrate_fp8(long long n, int B, long long bins, long long rows) {
  int saved[kNumFlags];
  CK(cudaStreamSynchronize(stream));
  CK(cudaMemcpy(saved, b_flags, sizeof saved, cudaMemcpyDeviceToHost));
  CK(cudaMemsetAsync(b_flags, 0, sizeof saved, stream));
  int rc = launch_pipeline(n, B, bins, rows, true);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h_flags, b_flags, sizeof saved, cudaMemcpyDeviceToHost, stream));
  int seg[kMaxS + 2];
  CK(cudaMemcpyAsync(seg, b_seg, sizeof(int) * (P.S + 1), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  CK(cudaMemcpy(b_flags, saved, sizeof saved, cudaMemcpyHostToDevice));
  const int st = check_flags();
  if (st) return st;
  bool all = true;
  for (int s = 0; s < P.S; ++s) {
    // species segments are padded to whole tiles, so a non-empty one has atoms
    if (seg[s + 1] > seg[s]) fp8_seen[s] = true;
    all = all && fp8_seen[s];
  }
  fp8_calibrated = all;
  fp8_pass_done = true;
  ++fp8_passes;
  return NNP_OK;
}

static void cross3(const double* u, const double* v, double* w) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}

// Cell steps cv_d (rows: B_d / nc_d, or ell_d along axis d) and their inverse.
void nnp::set_cell_steps(SysDesc& sd) {
  double M[9];
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c)
      M[3 * d + c] = sd.tric ? sd.B[3 * d + c] / sd.nc[d] : (c == d ? sd.ell[d] : 0.0);
  double r1r2[3], r2r0[3], r0r1[3];
  cross3(M + 3, M + 6, r1r2);
  cross3(M + 6, M, r2r0);
  cross3(M, M + 3, r0r1);
  const double det = M[0] * r1r2[0] + M[1] * r1r2[1] + M[2] * r1r2[2];
  const double* crs[3] = {r1r2, r2r0, r0r1};
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c) {
      sd.cv[3 * d + c] = sd.tric ? (float)M[3 * d + c] : (c == d ? sd.ellf[d] : 0.f);
      sd.cvinv[3 * c + d] = (float)(crs[d][c] / det);  // m_d = sum_c x_c cvinv[c][d]
    }
}

// Host-side set-up of the systems: cell grids, capacity, IO descriptor.
int nnp_ctx::prepare(int B, const int64_t* offsets, const double* pos_host_or_null,
                     const double* boxes, long long& bins, long long& rows) {
  sys_h.resize(B);
  long long cell_base = 0;
  const double rc = cfg.rc_r;
  for (int b = 0; b < B; ++b) {
    SysDesc& sd = sys_h[b];
    memset(&sd, 0, sizeof sd);
    sd.atom_begin = offsets[b];
    sd.atom_end = offsets[b + 1];
    const long long nb = sd.atom_end - sd.atom_begin;
    if (nb <= 0) return fail(NNP_ERR_INVALID_ARG, "system %d has %lld atoms", b, nb);
    double L[3];
    if (boxes) {
      const double* bx = boxes + 9 * (size_t)b;
      bool tric = false;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          if (!std::isfinite(bx[3 * r + c]))
            return fail(NNP_ERR_INVALID_ARG, "system %d: non-finite box entry", b);
          if (r != c && bx[3 * r + c] != 0.0) tric = true;
        }
      if (!tric) {
        for (int c = 0; c < 3; ++c) {
          L[c] = bx[4 * c];
          if (!(L[c] > 0.0)) return fail(NNP_ERR_INVALID_ARG, "system %d: box edge %d is %g", b, c, L[c]);
          if (L[c] < rc)
            return fail(NNP_ERR_UNSUPPORTED, "system %d: box edge %g is shorter than the radial cutoff %g",
                        b, L[c], rc);
        }
      } else {
        // rows are the cell vectors; cells are sized by the heights across them
        const double* u = bx;
        const double* v = bx + 3;
        const double* w = bx + 6;
        double vw[3], wu[3], uv[3];
        cross3(v, w, vw);
        cross3(w, u, wu);
        cross3(u, v, uv);
        const double V = u[0] * vw[0] + u[1] * vw[1] + u[2] * vw[2];
        if (!(V > 0.0)) return fail(NNP_ERR_INVALID_ARG, "system %d: the cell is not right-handed", b);
        const double* crs[3] = {vw, wu, uv};
        for (int d = 0; d < 3; ++d) {
          L[d] = V / std::sqrt(crs[d][0] * crs[d][0] + crs[d][1] * crs[d][1] + crs[d][2] * crs[d][2]);
          if (L[d] < rc)
            return fail(NNP_ERR_UNSUPPORTED, "system %d: cell height %g is shorter than the radial cutoff %g",
                        b, L[d], rc);
          for (int c = 0; c < 3; ++c) {
            sd.B[3 * d + c] = bx[3 * d + c];
            sd.Binv[3 * c + d] = crs[d][c] / V;  // s_d = sum_c r_c Binv[c][d]
          }
        }
        sd.tric = 1;
      }
      for (int c = 0; c < 3; ++c) sd.origin[c] = 0.0;
      sd.periodic = 1;
    } else {
      if (!pos_host_or_null) return fail(NNP_ERR_INVALID_ARG, "isolated system needs positions on the host");
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (long long a = sd.atom_begin; a < sd.atom_end; ++a)
        for (int c = 0; c < 3; ++c) {
          const double x = pos_host_or_null[3 * a + c];
          if (!std::isfinite(x)) return fail(NNP_ERR_INVALID_ARG, "non-finite position of atom %lld", a);
          lo[c] = std::min(lo[c], x);
          hi[c] = std::max(hi[c], x);
        }
      for (int c = 0; c < 3; ++c) {
        sd.origin[c] = lo[c] - 0.5;
        L[c] = hi[c] - lo[c] + 1.0;
      }
      sd.periodic = 0;
    }
    // cells of edge >= rc; no more than ~2 cells per atom in a system
    int nc[3];
    for (int c = 0; c < 3; ++c) nc[c] = std::max(1, (int)std::floor(L[c] / rc));
    const long long cap_cells = std::max<long long>(27, 2 * nb);
    while ((long long)nc[0] * nc[1] * nc[2] > cap_cells) {
      int c = (nc[0] >= nc[1] && nc[0] >= nc[2]) ? 0 : (nc[1] >= nc[2] ? 1 : 2);
      nc[c] = std::max(1, nc[c] * 3 / 4);
    }
    for (int c = 0; c < 3; ++c) {
      if (nc[c] > 1000) nc[c] = 1000;
      sd.L[c] = L[c];
      sd.nc[c] = nc[c];
      sd.ell[c] = L[c] / nc[c];
      sd.inv_L[c] = 1.0 / L[c];
      sd.inv_ell[c] = 1.0 / sd.ell[c];
      sd.ellf[c] = (float)sd.ell[c];
    }
    set_cell_steps(sd);
    sd.cell_base = (int)cell_base;
    cell_base += (long long)nc[0] * nc[1] * nc[2];
  }
  const long long n = offsets[B];
  bins = cell_base * P.S;
  rows = n + (long long)kTileRows * P.S;
  if (cell_base > (1ll << 30)) return fail(NNP_ERR_CAPACITY, "too many cells");
  if (n >= (1ll << 27)) return fail(NNP_ERR_CAPACITY, "at most 2^27 - 1 atoms per evaluation");
  total_cells = (int)cell_base;
  return NNP_OK;
}

int nnp_ctx::read_flags(int& fl_out) {
  (void)fl_out;
  return NNP_OK;
}

// One evaluation.  sync = true: wait, check flags, regrow lists and redo on
// overflow, copy results to host pointers.
int nnp_ctx::evaluate(int B, const int64_t* offsets, const double* pos, const int32_t* Z,
                      const double* boxes, double* energies, double* forces, bool sync) {
  if (!weights_ready()) return fail(NNP_ERR_NO_WEIGHTS, "weights missing for some species");
  if (B < 1 || !offsets || !pos || !Z) return fail(NNP_ERR_INVALID_ARG, "null argument or B < 1");
  if (offsets[0] != 0) return fail(NNP_ERR_INVALID_ARG, "offsets[0] must be 0");
  const long long n = offsets[B];
  if (n <= 0) return fail(NNP_ERR_INVALID_ARG, "no atoms");
  const bool pos_dev = is_device_ptr(pos), Z_dev = is_device_ptr(Z);
  const bool F_dev = forces && is_device_ptr(forces);
  const bool E_dev = energies && is_device_ptr(energies);
  if (!sync && (!pos_dev || !Z_dev || (forces && !F_dev) || (energies && !E_dev)))
    return fail(NNP_ERR_INVALID_ARG, "nnp_eval_async needs device pointers");
  std::vector<double> pos_tmp;
  const double* pos_host = pos_dev ? nullptr : pos;
  bool need_host_pos = false;
  if (!boxes) need_host_pos = true;
  if (need_host_pos && pos_dev) {
    pos_tmp.resize((size_t)n * 3);
    CK(cudaMemcpy(pos_tmp.data(), pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    pos_host = pos_tmp.data();
  }
  long long bins = 0, rows = 0;
  int rc = prepare(B, offsets, pos_host, boxes, bins, rows);
  if (rc) return rc;
  for (int attempt = 0; attempt < 4; ++attempt) {
    rc = ensure_capacity(n, B, bins, rows);
    if (rc) return rc;
    // IO and system descriptors through the next pinned staging slot
    Stage& sg = stages[stage_next];
    stage_next = (stage_next + 1) % kStages;
    CK(cudaEventSynchronize(sg.ev));  // the copies that last read this slot have run
    if (sg.cap < (size_t)B) {
      if (sg.sys) cudaFreeHost(sg.sys);
      sg.sys = nullptr;
      sg.cap = 0;
      CK(cudaMallocHost(&sg.sys, sizeof(SysDesc) * (size_t)B));
      sg.cap = (size_t)B;
    }
    memcpy(sg.sys, sys_h.data(), sizeof(SysDesc) * (size_t)B);
    h_io = sg.io;
    EvalIO& io = *sg.io;
    // page-locked host inputs are read in place by the binning kernel (the
    // only reader of positions and species outside the pair-list and
    // embedding modes): on the B300 host links measured here, SM loads move
    // them faster than a host-to-device DMA copy of these sizes
    const bool in_place = !ext_mode && !ee_mode;
    const double* pos_map = (!pos_dev && in_place) ? static_cast<const double*>(mapped_host_ptr(pos)) : nullptr;
    const int32_t* Z_map = (!Z_dev && in_place) ? static_cast<const int32_t*>(mapped_host_ptr(Z)) : nullptr;
    io.pos = pos_dev ? pos : (pos_map ? pos_map : b_pos_stage);
    io.Z = Z_dev ? Z : (Z_map ? Z_map : b_Z_stage);
    io.forces = F_dev ? forces : b_F_stage;
    io.energies = E_dev ? energies : b_E_stage;
    io.n_atoms = n;
    io.n_sys = B;
    io.total_cells = total_cells;
    io.pairs = ext_pairs;
    io.shifts = ext_shifts;
    io.n_pairs = ext_n_pairs;
    if (!pos_dev && !pos_map)
      CK(cudaMemcpyAsync(b_pos_stage, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, stream));
    if (!Z_dev && !Z_map) CK(cudaMemcpyAsync(b_Z_stage, Z, sizeof(int) * n, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_io, sg.io, sizeof(EvalIO), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(b_sys, sg.sys, sizeof(SysDesc) * B, cudaMemcpyHostToDevice, stream));
    CK(cudaEventRecord(sg.ev, stream));
    // device flags accumulate over asynchronous evaluations until nnp_sync reads them;
    // a synchronous evaluation reports only its own
    if (sync) CK(cudaMemsetAsync(b_flags, 0, sizeof(int) * kNumFlags, stream));
    if (cfg.precision == NNP_FP8 && !fp8_pass_done) {
      rc = calibrate_fp8(n, B, bins, rows);
      if (rc == -1) continue;  // lists regrown: evaluate again
      if (rc) return rc;
    }
    if ((cfg.flags & NNP_FLAG_AUTOTUNE) && sync) {
      rc = autotune(n, B, bins, rows);
      if (rc) return rc;
    }
    const bool use_graph = !(cfg.flags & NNP_FLAG_NO_GRAPH);
    if (use_graph) {
      const int ext = ext_mode ? 1 : 0;
      const long long eek = ee_mode ? ee_n_mm : -1;
      if (!gexec || g_key_n != n || g_key_B != B || g_key_bins != bins || g_key_ext != ext || g_key_ee != eek) {
        invalidate_graph();
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        int lrc = launch_pipeline(n, B, bins, rows);
        cudaError_t ce = cudaStreamEndCapture(stream, &graph);
        if (lrc) { if (ce == cudaSuccess) cudaGraphDestroy(graph); return lrc; }
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        ce = cudaGraphInstantiate(&gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) { gexec = nullptr; return cuda_fail(ce, "cudaGraphInstantiate"); }
        g_key_n = n; g_key_B = B; g_key_bins = bins; g_key_ext = ext; g_key_ee = eek;
        ++graph_captures;
      }
      CK(cudaGraphLaunch(gexec, stream));
    } else {
      rc = launch_pipeline(n, B, bins, rows);
      if (rc) return rc;
    }
    last_n = n; last_B = B; last_rows = rows; has_state = true;
    CK(cudaMemcpyAsync(h_flags, b_flags, sizeof(int) * kNumFlags, cudaMemcpyDeviceToHost, stream));
    if (!sync) return NNP_OK;
    // results to host buffers on the stream, so that one synchronisation
    // covers them; if the flags ask for a regrow they are overwritten below
    if (forces && !F_dev)
      CK(cudaMemcpyAsync(forces, b_F_stage, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, stream));
    if (energies && !E_dev)
      CK(cudaMemcpyAsync(energies, b_E_stage, sizeof(double) * B, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    int st = check_flags();
    if (st == -1) continue;  // lists regrown: evaluate again
    if (st) return st;
    return NNP_OK;
  }
  return fail(NNP_ERR_CAPACITY, "neighbour lists still overflow after regrowing");
}

// Returns 0, an error code, or -1 if the lists were regrown (caller redoes).
int nnp_ctx::check_flags() {
  const int* f = h_flags;
  max_nbr_r = f[kFlagMaxNbrR];
  max_nbr_a = f[kFlagMaxNbrA];
  if (f[kFlagNonFinite]) return fail(NNP_ERR_INVALID_ARG, "non-finite atom position");
  if (f[kFlagBadSpecies]) return fail(NNP_ERR_UNKNOWN_SPECIES, "atomic number outside the configured species");
  if (f[kFlagTimeout]) return fail(NNP_ERR_TIMEOUT, "a bounded device wait expired (tensor-core network)");
  if (f[kFlagBadPair])
    return fail(NNP_ERR_INVALID_ARG, "pair list: an index is out of range or a shift is not a whole periodic image");
  if (f[kFlagChecked])
    return fail(NNP_ERR_BOUNDS, "bounds check: index %d out of range at source line %d", f[kFlagCheckedValue],
                f[kFlagCheckedLine]);
  if (f[kFlagFp8Uncal]) {  // FP8: a species without activation ranges: calibrate and evaluate again
    fp8_pass_done = false;
    return -1;
  }
  if (f[kFlagOverflowR] || f[kFlagOverflowA]) {
    if (f[kFlagOverflowR]) cap_r = ((int)(f[kFlagMaxNbrR] * 1.25) + 31) / 32 * 32;
    if (f[kFlagOverflowA]) cap_a = ((int)(f[kFlagMaxNbrA] * 1.25) + 15) / 16 * 16;
    // the descriptor backward parks every angular pair of a row in shared memory
    if (cap_r > kMaxCapR || cap_a > kMaxCapA)
      return fail(NNP_ERR_CAPACITY, "neighbour counts too large (%d radial, %d angular)",
                  f[kFlagMaxNbrR], f[kFlagMaxNbrA]);
    invalidate_graph();
    return -1;
  }
  return NNP_OK;
}

bool nnp_ctx::charges_ready() const {
  if (!has_charges) return false;
  for (int s = 0; s < P.S; ++s)
    if (!has_w[(size_t)n_members * kMaxS + s]) return false;
  return true;
}

bool nnp_ctx::weights_ready() const {
  for (int s = 0; s < P.S; ++s)
    for (int m = 0; m < n_members; ++m)
      if (!has_w[(size_t)m * kMaxS + s]) return false;
  return true;
}

// ---------------------------------------------------------------------------
// C ABI

namespace nnp {
// NNP_SELFTEST_BOUNDS: one index that is out of range, through the checked build's check
__global__ void k_bounds_selftest(int* flags) {
  if (threadIdx.x == 0) (void)NNP_IN(7, 3, flags);  // the check records the index
}
}  // namespace nnp

extern "C" {

int nnp_config_init(nnp_config* cfg, int32_t n_species, const int32_t* atomic_numbers) {
  if (!cfg || n_species < 1 || n_species > NNP_MAX_SPECIES || !atomic_numbers) return NNP_ERR_INVALID_ARG;
  for (int s = 1; s < n_species; ++s)
    if (atomic_numbers[s] <= atomic_numbers[s - 1]) return NNP_ERR_INVALID_ARG;
  memset(cfg, 0, sizeof *cfg);
  cfg->n_species = n_species;
  for (int s = 0; s < n_species; ++s) cfg->atomic_numbers[s] = atomic_numbers[s];
  cfg->rc_r = 5.2;
  cfg->eta_r = 16.0;
  cfg->n_rad = 16;
  for (int m = 0; m < 16; ++m) cfg->shf_r[m] = 0.9 + 0.26875 * m;
  cfg->rc_a = 3.5;
  cfg->eta_a = 8.0;
  cfg->zeta = 32.0;
  cfg->n_ang_r = 4;
  cfg->n_ang_z = 8;
  for (int a = 0; a < 4; ++a) cfg->shf_a[a] = 0.9 + 0.65 * a;
  for (int z = 0; z < 8; ++z) cfg->shf_z[z] = (2 * z + 1) * 3.14159265358979323846 / 16.0;
  cfg->hidden[0] = 160;
  cfg->hidden[1] = 128;
  cfg->hidden[2] = 96;
  cfg->celu_alpha = 0.1;
  cfg->precision = NNP_FP32;
  cfg->max_atoms = 4096;
  cfg->max_systems = 1;
  cfg->nbr_capacity = 0;
  cfg->ang_capacity = 0;
  cfg->stream = nullptr;
  cfg->flags = 0;
  return NNP_OK;
}

int nnp_create(const nnp_config* cfg, nnp_ctx** out) {
  if (!out) return NNP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg) { g_create_error = "null config"; return NNP_ERR_INVALID_ARG; }
  auto bad = [&](int code, const char* msg) { g_create_error = msg; return code; };
  const int S = cfg->n_species;
  if (S < 1 || S > NNP_MAX_SPECIES) return bad(NNP_ERR_INVALID_ARG, "n_species outside 1..8");
  if (S > kMaxS) return bad(NNP_ERR_UNSUPPORTED, "the kernels support at most 8 species");
  for (int s = 0; s < S; ++s) {
    if (cfg->atomic_numbers[s] < 1 || cfg->atomic_numbers[s] > 127)
      return bad(NNP_ERR_INVALID_ARG, "atomic numbers must lie in 1..127");
    if (s && cfg->atomic_numbers[s] <= cfg->atomic_numbers[s - 1])
      return bad(NNP_ERR_INVALID_ARG, "atomic numbers must be ascending");
  }
  if (cfg->n_rad != kNRad || cfg->n_ang_r != kNAngR || cfg->n_ang_z != kNAngZ)
    return bad(NNP_ERR_UNSUPPORTED, "kernels are specialised for 16 radial, 4 x 8 angular terms");
  if (cfg->hidden[0] != kH1 || cfg->hidden[1] != kH2 || cfg->hidden[2] != kH3)
    return bad(NNP_ERR_UNSUPPORTED, "kernels are specialised for hidden widths 160/128/96");
  if (!(cfg->rc_r > 0) || !(cfg->rc_a > 0) || cfg->rc_a > cfg->rc_r)
    return bad(NNP_ERR_INVALID_ARG, "cutoffs must satisfy 0 < rc_a <= rc_r");
  int zsq = -1;
  for (int q = 0; q <= 6; ++q)
    if (cfg->zeta == (double)(1 << q)) zsq = q;
  if (zsq < 0) return bad(NNP_ERR_UNSUPPORTED, "zeta must be a power of two <= 64");
  if (!(cfg->celu_alpha > 0)) return bad(NNP_ERR_INVALID_ARG, "celu_alpha must be positive");
  if (cfg->precision < NNP_FP32 || cfg->precision > NNP_FP8)
    return bad(NNP_ERR_INVALID_ARG, "unknown precision");
  if (cfg->n_members < 0) return bad(NNP_ERR_INVALID_ARG, "negative ensemble size");
  const int members = cfg->n_members > 0 ? cfg->n_members : 1;
  if (members > NNP_MAX_MEMBERS) return bad(NNP_ERR_INVALID_ARG, "at most NNP_MAX_MEMBERS ensemble members");
  if ((cfg->flags & NNP_FLAG_CHARGES) && cfg->precision == NNP_FP8)
    return bad(NNP_ERR_UNSUPPORTED, "the FP8 form has no charge network");

  nnp_ctx* c = new nnp_ctx();
  c->cfg = *cfg;
  DescParams& P = c->P;
  P.S = S;
  P.D = kNRad * S + kNAng * S * (S + 1) / 2;
  P.zeta_sq = zsq;
  P.rc_r = (float)cfg->rc_r;
  P.eta_r = (float)cfg->eta_r;
  P.rc_a = (float)cfg->rc_a;
  P.eta_a = (float)cfg->eta_a;
  for (int m = 0; m < kNRad; ++m) P.shf_r[m] = (float)cfg->shf_r[m];
  {
    const double dR = cfg->shf_r[1] - cfg->shf_r[0];
    bool even = dR > 0.0;
    for (int m = 0; m < kNRad; ++m)
      even = even && std::fabs(cfg->shf_r[m] - (cfg->shf_r[0] + m * dR)) <= 1e-6 * (1.0 + std::fabs(cfg->shf_r[m]));
    P.rad_even = even ? 1 : 0;
    P.rad_gk = (float)(2.0 * cfg->eta_r * dR / std::log(2.0));
    for (int d = 1; d <= 4; ++d) P.rad_c[d - 1] = (float)std::exp(-cfg->eta_r * dR * dR * (2 * d - 1));
  }
  for (int a = 0; a < kNAngR; ++a) P.shf_a[a] = (float)cfg->shf_a[a];
  for (int z = 0; z < kNAngZ; ++z) {
    P.hcos_z[z] = (float)(0.5 * std::cos(cfg->shf_z[z]));
    P.hsin_z[z] = (float)(0.5 * std::sin(cfg->shf_z[z]));
  }
  P.celu_alpha = (float)cfg->celu_alpha;
  c->cap_r = cfg->nbr_capacity > 0 ? cfg->nbr_capacity : 96;
  c->cap_a = cfg->ang_capacity > 0 ? cfg->ang_capacity : 32;
  c->n_members = members;
  c->has_charges = (cfg->flags & NNP_FLAG_CHARGES) != 0;
  int rc = c->init_device();
  if (!rc) rc = noalloc_prepare(c);
  if (rc) {
    g_create_error = c->err;
    delete c;
    return rc;
  }
  *out = c;
  return NNP_OK;
}

void nnp_destroy(nnp_ctx* ctx) { delete ctx; }

const char* nnp_last_error(const nnp_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

int nnp_set_weights(nnp_ctx* ctx, int32_t species, const float* const W[4], const float* const b[4]) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (species < 0 || species >= ctx->P.S) return ctx->fail(NNP_ERR_INVALID_ARG, "species index %d", species);
  if (!W || !b) return ctx->fail(NNP_ERR_INVALID_ARG, "null weight arrays");
  for (int l = 0; l < 4; ++l)
    if (!W[l] || !b[l]) return ctx->fail(NNP_ERR_INVALID_ARG, "null weight or bias of layer %d", l);
  return ctx->set_weights(0, species, W, b);
}

int nnp_set_member_weights(nnp_ctx* ctx, int32_t member, int32_t species, const float* const W[4],
                           const float* const b[4]) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (member < 0 || member >= ctx->n_members) return ctx->fail(NNP_ERR_INVALID_ARG, "member index %d", member);
  if (species < 0 || species >= ctx->P.S) return ctx->fail(NNP_ERR_INVALID_ARG, "species index %d", species);
  if (!W || !b) return ctx->fail(NNP_ERR_INVALID_ARG, "null weight arrays");
  for (int l = 0; l < 4; ++l)
    if (!W[l] || !b[l]) return ctx->fail(NNP_ERR_INVALID_ARG, "null weight or bias of layer %d", l);
  return ctx->set_weights(member, species, W, b);
}

int nnp_eval(nnp_ctx* ctx, int64_t n, const double* pos, const int32_t* Z, const double* box,
             double* energy, double* forces) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (n <= 0) return ctx->fail(NNP_ERR_INVALID_ARG, "n must be positive");
  int64_t off[2] = {0, n};
  return ctx->evaluate(1, off, pos, Z, box, energy, forces, true);
}

int nnp_eval_pairs(nnp_ctx* ctx, int64_t n, const double* pos, const int32_t* Z, const double* box,
                   int64_t n_pairs, const int32_t* pairs, const double* shifts, double* energy, double* forces) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (n <= 0) return ctx->fail(NNP_ERR_INVALID_ARG, "n must be positive");
  if (n_pairs < 0 || (n_pairs > 0 && !pairs)) return ctx->fail(NNP_ERR_INVALID_ARG, "null pair list");
  if (!box && shifts) return ctx->fail(NNP_ERR_INVALID_ARG, "shifts need a periodic box");
  const int* d_pairs = pairs;
  const double* d_shifts = shifts;
  cudaError_t e = cudaSuccess;
  const size_t np = (size_t)(n_pairs > 0 ? n_pairs : 1);
  if (n_pairs > 0 && !is_device_ptr(pairs)) {
    e = grow(ctx->b_pairs_stage, ctx->c_pairs_stage, 2 * np);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->b_pairs_stage, pairs, sizeof(int) * 2 * n_pairs, cudaMemcpyHostToDevice, ctx->stream);
    d_pairs = ctx->b_pairs_stage;
  }
  if (e == cudaSuccess && shifts && n_pairs > 0 && !is_device_ptr(shifts)) {
    e = grow(ctx->b_shifts_stage, ctx->c_shifts_stage, 3 * np);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->b_shifts_stage, shifts, sizeof(double) * 3 * n_pairs, cudaMemcpyHostToDevice,
                          ctx->stream);
    d_shifts = ctx->b_shifts_stage;
  }
  if (e != cudaSuccess) return ctx->cuda_fail(e, "nnp_eval_pairs staging");
  // an empty list still selects the pair-list path (no neighbours at all)
  ctx->ext_mode = true;
  ctx->ext_pairs = n_pairs > 0 ? d_pairs : nullptr;
  ctx->ext_shifts = n_pairs > 0 ? d_shifts : nullptr;
  ctx->ext_n_pairs = n_pairs;
  int64_t off[2] = {0, n};
  const int rc = ctx->evaluate(1, off, pos, Z, box, energy, forces, true);
  ctx->ext_mode = false;
  ctx->ext_pairs = nullptr;
  ctx->ext_shifts = nullptr;
  ctx->ext_n_pairs = 0;
  return rc;
}

int nnp_eval_async(nnp_ctx* ctx, int64_t n, const double* pos, const int32_t* Z, const double* box,
                   double* energy, double* forces) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (n <= 0) return ctx->fail(NNP_ERR_INVALID_ARG, "n must be positive");
  if (!box) return ctx->fail(NNP_ERR_INVALID_ARG, "nnp_eval_async needs a periodic box");
  int64_t off[2] = {0, n};
  return ctx->evaluate(1, off, pos, Z, box, energy, forces, false);
}

int nnp_sync(nnp_ctx* ctx) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaStreamSynchronize");
  if (!ctx->has_state) return NNP_OK;
  e = cudaMemcpy(ctx->h_flags, ctx->b_flags, sizeof(int) * kNumFlags, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(ctx->b_flags, 0, sizeof(int) * kNumFlags);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "nnp_sync flags");
  const bool uncal = ctx->h_flags[kFlagFp8Uncal] != 0;
  int st = ctx->check_flags();
  if (st == -1 && uncal)
    return ctx->fail(NNP_ERR_NO_WEIGHTS,
                     "FP8: a species appeared that no calibration pass has seen; the next evaluation calibrates, "
                     "evaluate again");
  if (st == -1)
    return ctx->fail(NNP_ERR_CAPACITY,
                     "neighbour lists overflowed since the last check; capacity grown, evaluate again");
  return st;
}

int nnp_eval_batch(nnp_ctx* ctx, int32_t B, const int64_t* offsets, const double* pos, const int32_t* Z,
                   const double* boxes, double* energies, double* forces) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (B < 1 || !offsets) return ctx->fail(NNP_ERR_INVALID_ARG, "B < 1 or null offsets");
  for (int b = 0; b < B; ++b)
    if (offsets[b + 1] <= offsets[b]) return ctx->fail(NNP_ERR_INVALID_ARG, "offsets must increase");
  return ctx->evaluate(B, offsets, pos, Z, boxes, energies, forces, true);
}

int nnp_eval_batch_async(nnp_ctx* ctx, int32_t B, const int64_t* offsets, const double* pos, const int32_t* Z,
                         const double* boxes, double* energies, double* forces) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (B < 1 || !offsets) return ctx->fail(NNP_ERR_INVALID_ARG, "B < 1 or null offsets");
  if (!boxes) return ctx->fail(NNP_ERR_INVALID_ARG, "nnp_eval_batch_async needs periodic boxes");
  for (int b = 0; b < B; ++b)
    if (offsets[b + 1] <= offsets[b]) return ctx->fail(NNP_ERR_INVALID_ARG, "offsets must increase");
  return ctx->evaluate(B, offsets, pos, Z, boxes, energies, forces, false);
}

int64_t nnp_param_count(const nnp_ctx* ctx) {
  if (!ctx) return -1;
  const int64_t D = ctx->P.D;
  return (int64_t)ctx->n_members * ctx->P.S * (D * kH1 + kH1 + kH1 * kH2 + kH2 + kH2 * kH3 + kH3 + kH3 + 1);
}

int nnp_force_match_grad(nnp_ctx* ctx, const double* v, const double* Fref, double* loss, double* grad) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  return ctx->force_match_grad(v, Fref, loss, grad);
}

int nnp_query(nnp_ctx* ctx, int32_t key, int64_t* value) {
  if (!ctx || !value) return NNP_ERR_INVALID_ARG;
  switch (key) {
    case NNP_Q_LAUNCHES_PER_EVAL: *value = ctx->launches_per_eval; break;
    case NNP_Q_NBR_CAPACITY: *value = ctx->cap_r; break;
    case NNP_Q_ANG_CAPACITY: *value = ctx->cap_a; break;
    case NNP_Q_MAX_NBR: *value = ctx->max_nbr_r; break;
    case NNP_Q_MAX_ANG: *value = ctx->max_nbr_a; break;
    case NNP_Q_ROWS: *value = ctx->last_rows; break;
    case NNP_Q_GRAPH_CAPTURES: *value = ctx->graph_captures; break;
    case NNP_Q_TUNE_NEIGHBOURS: *value = ctx->tune.nbr; break;
    case NNP_Q_TUNE_DESCRIPTOR: *value = ctx->tune.fwd; break;
    case NNP_Q_TUNE_BACKWARD: *value = ctx->tune.bwd; break;
    case NNP_Q_FP8_CALIBRATED: *value = ctx->fp8_calibrated ? 1 : 0; break;
    case NNP_Q_TUNE_DESCRIPTOR_TILE: *value = ctx->tune.fwd_tile; break;
    case NNP_Q_TUNE_BACKWARD_TILE: *value = ctx->tune.bwd_tile; break;
    case NNP_Q_TUNE_NEIGHBOURS_QUEUE: *value = ctx->tune.nbr_dyn; break;
#ifdef NNP_CHECKED
    case NNP_Q_CHECKED_BUILD: *value = 1; break;
#else
    case NNP_Q_CHECKED_BUILD: *value = 0; break;
#endif
    case NNP_Q_FP8_PASSES: *value = ctx->fp8_passes; break;
    default: return ctx->fail(NNP_ERR_INVALID_ARG, "unknown query key %d", key);
  }
  return NNP_OK;
}

int nnp_atom_energies(nnp_ctx* ctx, double* out) {
  if (!ctx || !out) return NNP_ERR_INVALID_ARG;
  if (!ctx->has_state) return ctx->fail(NNP_ERR_NO_STATE, "no evaluation yet");
  const long long rows = ctx->last_rows;
  std::vector<int> ra((size_t)rows);
  std::vector<float> ei((size_t)rows);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpy(ra.data(), ctx->b_row_atom, sizeof(int) * rows, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ei.data(), ctx->b_Ei, sizeof(float) * rows, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "nnp_atom_energies copy");
  int seg[kMaxS + 2];
  e = cudaMemcpy(seg, ctx->b_seg, sizeof(seg), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "nnp_atom_energies copy");
  const long long used = seg[ctx->P.S];
  for (long long r = 0; r < used && r < rows; ++r)
    if (ra[r] >= 0 && ra[r] < ctx->last_n) out[ra[r]] = (double)ei[r];
  return NNP_OK;
}

int nnp_selftest(nnp_ctx* ctx, int32_t test) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (test != NNP_SELFTEST_WAIT_TIMEOUT && test != NNP_SELFTEST_BOUNDS)
    return ctx->fail(NNP_ERR_INVALID_ARG, "unknown self-test %d", test);
  int f[kNumFlags];
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->b_flags, 0, sizeof f, ctx->stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "nnp_selftest");
  if (test == NNP_SELFTEST_BOUNDS) {
    k_bounds_selftest<<<1, 32, 0, ctx->stream>>>(ctx->b_flags);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, ctx->b_flags, sizeof f, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->b_flags, 0, sizeof f, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "nnp_selftest");
    if (f[kFlagChecked])
      return ctx->fail(NNP_ERR_BOUNDS, "self-test: index %d out of range was caught (line %d), as designed",
                       f[kFlagCheckedValue], f[kFlagCheckedLine]);
    return ctx->fail(NNP_ERR_UNSUPPORTED, "self-test: the library was built without NNP_CHECKED");
  }
  launch_wait_selftest(ctx->stream, ctx->b_flags, 2000000ull);  // 2 ms
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, ctx->b_flags, sizeof f, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->b_flags, 0, sizeof f, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "nnp_selftest");
  if (f[kFlagTimeout]) return ctx->fail(NNP_ERR_TIMEOUT, "self-test: the bounded wait expired and returned, as designed");
  return ctx->fail(NNP_ERR_CUDA, "self-test: a wait on a barrier that nothing completes did not time out");
}

int nnp_profile_force_match(nnp_ctx* ctx, double* out, int32_t n_out) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (!out || n_out < 0) return ctx->fail(NNP_ERR_INVALID_ARG, "null output");
  return ctx->profile_force_match(out, n_out);
}

int nnp_profile_stages(nnp_ctx* ctx, double* out, int32_t n_out) {
  if (!ctx || !out) return NNP_ERR_INVALID_ARG;
  return ctx->profile_stages(out, n_out);
}

}  // extern "C"
