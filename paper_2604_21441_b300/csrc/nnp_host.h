// nnp_host.h -- the context object behind the C ABI and the kernel launch
// entry points shared between the host translation units.
#pragma once
#include <string>
#include <vector>

#include "../../include/nnp.h"
#include "nnp_internal.cuh"

namespace nnp {

// k_cells.cu
__global__ void k_bin(const EvalIO* io, const SysDesc* sys, const signed char* zlut, Workspace ws);
__global__ void k_scan(const EvalIO* io, int S, Workspace ws);
__global__ void k_scatter(const EvalIO* io, Workspace ws);
__global__ void k_binsort(const EvalIO* io, int S, int sort, Workspace ws);
// the four above in one block of 1024 threads (at most kCellsRowsSmall rows);
// dynamic shared memory sizeof(int) * kScanSmemBins
__global__ void k_cells_small(const EvalIO* io, const SysDesc* sys, const signed char* zlut, int S, int sort,
                              Workspace ws);
// grid: blocks for a warp per cell, or (mode & 2) per half cell, for systems
// above kNbrRowsSmall rows; rows and cells (totals over systems) choose the
// small-system form and its split.  mode bit 0: items from the work queue
// instead of static order; bit 1: each cell's row groups of 16 alternate
// between two warps (large systems only; cells of many rows)
void launch_neighbors(int grid, cudaStream_t st, const EvalIO* io, const SysDesc* sys, const DescParams& P,
                      const Workspace& ws, long long rows, long long cells, int nsm, int mode = 0);
void set_cell_steps(SysDesc& sd);  // cell steps and their inverse from nc, ell or B
void launch_wait_selftest(cudaStream_t st, int* flags, unsigned long long limit_ns);
__global__ void k_pairs_prep(int S, Workspace ws);
__global__ void k_pairs_count(const EvalIO* io, const SysDesc* sys, DescParams P, Workspace ws);
__global__ void k_pairs_offsets(const EvalIO* io, int S, Workspace ws, int* cur);
__global__ void k_pairs_fill(const EvalIO* io, const SysDesc* sys, DescParams P, Workspace ws, int* cur);
size_t neighbors_smem(int win);
cudaError_t neighbors_set_smem_limits();

// k_aev.cu
// rows: upper bound of the rows of the evaluation (grid sizing only)
// per_sm: cap on resident blocks per SM of the grid (0 = built-in default)
void launch_aev_fwd(long long rows, int nsm, cudaStream_t st, const SysDesc* sys, const DescParams& P,
                    const Workspace& ws, int mode /* GMode */, int per_sm = 0, int tile = 0);
// k_aev_bwd: forces accumulate in FP64 straight into io->forces (zeroed
// by k_bin)
void launch_aev_bwd(long long rows, int nsm, cudaStream_t st, const EvalIO* io, const SysDesc* sys,
                    const DescParams& P, const Workspace& ws, int per_sm = 0, int tile = 0);
cudaError_t aev_set_smem_limits();

// k_mlp_f32.cu
void launch_mlp_f32(int grid, cudaStream_t st, const EvalIO* io, const DescParams& P,
                    const Workspace& ws, const MlpF32Weights& W, int acc = 0);
cudaError_t mlp_f32_set_smem_limits();
void launch_fm(int grid, cudaStream_t st, const DescParams& P, const Workspace& ws, const MlpF32Weights& W,
               const float* dG, float* z, float* dz, float* t, float* p);
void launch_fm_wgrad(int grid, cudaStream_t st, const DescParams& P, const FmJob* jobs, int njobs,
                     const float* G, const float* dG, const float* z, const float* dz, const float* t,
                     const float* p, double* grad);
void launch_aev_jvp(long long rows, int nsm, cudaStream_t st, const SysDesc* sys, const DescParams& P,
                    const Workspace& ws, const double* v, float* dG);

}  // namespace nnp

struct nnp_ctx;
namespace nnp {
// k_mlp_tc.cu (tensor-core network); returns an nnp_status
// io / ws: the network's I/O block and workspace (null: the context's own)
// Members m0 .. m0 + nm - 1 side by side; accm = 1 adds E_i and dE/dG with
// reductions (the caller zeroes them first), 0 writes them.
int launch_mlp_tc(nnp_ctx* ctx, cudaStream_t st, long long rows, int m0, int nm, int accm,
                  const EvalIO* io = nullptr, const Workspace* ws = nullptr);
int mlp_tc_init(nnp_ctx* ctx);
int noalloc_prepare(nnp_ctx* ctx);  // nnp_create: scratch address and kernels of nnp_eval_noalloc
int mlp_tc_set_weights(nnp_ctx* ctx, int member, int species, const float* host_blob);
int launch_fp8_calib(nnp_ctx* ctx, cudaStream_t st, long long rows);
void mlp_tc_free(nnp_ctx* ctx);
}  // namespace nnp

struct nnp_ctx {
  nnp_config cfg{};
  nnp::DescParams P{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 148;
  std::string err;

  // capacities
  int cap_r = 96, cap_a = 32;
  int total_cells = 0;

  // device buffers (capacity in elements)
  int *b_bin_count = nullptr, *b_bin_start = nullptr, *b_bin_len = nullptr;
  size_t c_bins = 0, c_bins1 = 0, c_bins2 = 0;
  int *b_atom_bin = nullptr, *b_atom_slot = nullptr, *b_atom_cell = nullptr, *b_atom_sys = nullptr;
  float4* b_atom_off = nullptr;
  size_t c_atoms1 = 0, c_atoms2 = 0, c_atoms3 = 0, c_atoms4 = 0, c_atoms5 = 0;
  int *b_row_atom = nullptr, *b_row_info = nullptr, *b_row_cell = nullptr;
  float4* b_pos4 = nullptr;
  size_t c_rows1 = 0, c_rows2 = 0, c_rows3 = 0, c_rows4 = 0, c_rows5 = 0, c_rows6 = 0;
  int *b_cnt_r = nullptr, *b_cnt_a = nullptr, *b_nbr_r = nullptr;
  size_t c_nbr_r = 0;
  float *b_G = nullptr, *b_dEdG = nullptr, *b_Ei = nullptr;
  __nv_bfloat16* b_Gh = nullptr;
  size_t c_G = 0, c_Gh = 0, c_dEdG = 0, c_Ei = 0;
  // tensor-core ensembles of wide networks: every (tile, member)'s g1 tile, so that
  // dE/dG is one product over all members (ens_wide())
  uint8_t* b_g1 = nullptr;
  size_t c_g1 = 0;
  bool ens_wide() const {
    return cfg.precision != NNP_FP32 && n_members > 1 && P.D != 128 && P.D != 48;
  }
  nnp::SysDesc* b_sys = nullptr;
  size_t c_sys = 0;
  double* b_pos_stage = nullptr;
  int* b_Z_stage = nullptr;
  double *b_F_stage = nullptr, *b_E_stage = nullptr;
  size_t c_pos_stage = 0, c_Z_stage = 0, c_F_stage = 0, c_E_stage = 0;
  int* b_seg = nullptr;
  int* b_flags = nullptr;
  int* b_queue = nullptr;       // work-queue counters (Workspace::queue)
  signed char* d_zlut = nullptr;
  nnp::EvalIO* d_io = nullptr;
  nnp::EvalIO* h_io = nullptr;  // pinned; the staging slot of the last evaluation
  // Pinned staging slots for the per-call descriptors, used in turn: a slot is
  // rewritten only after the copies that read it (event) have run, so
  // asynchronous evaluations never wait for the stream.
  static constexpr int kStages = 4;
  struct Stage {
    nnp::EvalIO* io = nullptr;
    nnp::SysDesc* sys = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
  } stages[kStages];
  int stage_next = 0;
  int* h_flags = nullptr;       // pinned

  // weights
  float* b_wf32 = nullptr;      // FP32 blob, all species
  size_t wf32_stride = 0;       // floats per species
  nnp::MlpF32Weights wf32{};                 // ensemble member 0 (every single-network path)
  int n_members = 1;                         // networks averaged per species (ensemble)
  std::vector<nnp::MlpF32Weights> wf32m;     // per member; wf32m[0] == wf32
  std::vector<unsigned char> has_w;          // [member * kMaxS + species]
  std::vector<float> host_weights;  // FP32 copy (layout of nnp_param_count), for re-quantisation
  void* tc = nullptr;           // tensor-core network state (k_mlp_tc.cu)
  int* b_q8 = nullptr;          // FP8 scales (Workspace::q8)
  bool fp8_calibrated = false;  // every species has been seen by a calibration pass
  bool fp8_pass_done = false;   // a calibration pass has run since the weights were set
  long long fp8_passes = 0;     // calibration passes run
  bool fp8_seen[nnp::kMaxS] = {};
  int calibrate_fp8(long long n, int B, long long bins, long long rows);

  // force-matching buffers (allocated on first use)
  float *fm_z = nullptr, *fm_dz = nullptr, *fm_t = nullptr, *fm_p = nullptr;
  double *fm_v = nullptr, *fm_ref = nullptr, *fm_grad = nullptr;
  nnp::FmJob* fm_jobs = nullptr;
  std::vector<nnp::FmJob> fm_job_list;  // host copy of fm_jobs, built for the segments fm_job_seg
  int fm_job_seg[nnp::kMaxS + 2] = {};
  size_t fm_cap = 0, fm_cap2 = 0, fm_cap3 = 0, fm_cap4 = 0, fm_vcap = 0, fm_refcap = 0, fm_gcap = 0, fm_jcap = 0;
  static bool is_device(const void* p);

  // caller's pair list for the current evaluation (nnp_eval_pairs; device
  // pointers, null otherwise) and the per-row fill cursors it needs
  bool ext_mode = false;
  const int* ext_pairs = nullptr;
  const double* ext_shifts = nullptr;
  long long ext_n_pairs = 0;
  int* b_pair_cur = nullptr;
  int* b_pairs_stage = nullptr;
  double* b_shifts_stage = nullptr;
  size_t c_pair_cur = 0, c_pairs_stage = 0, c_shifts_stage = 0;
  int g_key_ext = -1;

  // electrostatic embedding (nnp_ee.cu; NNP_FLAG_CHARGES): the charge
  // network is weight set n_members; buffers are allocated on first use
  bool has_charges = false;
  bool ee_mode = false;          // the current evaluation embeds
  long long ee_n_ml = 0, ee_n_mm = 0;
  long long g_key_ee = -1;
  nnp::EeIO* h_ee = nullptr;     // pinned
  nnp::EeIO* d_ee = nullptr;
  nnp::EvalIO* d_io_q = nullptr; // the charge pass's I/O block
  float4 *b_ee_mmhi = nullptr, *b_ee_mmlo = nullptr, *b_ee_mlhi = nullptr, *b_ee_mllo = nullptr;
  double *b_ee_V = nullptr, *b_ee_field = nullptr, *b_ee_qatom = nullptr, *b_ee_qout = nullptr;
  double *b_ee_mmF = nullptr, *b_ee_mmpos = nullptr, *b_ee_mmq = nullptr, *b_ee_sums = nullptr;
  float *b_ee_qrows = nullptr, *b_ee_dqdG = nullptr;
  size_t c_ee_n = 0, c_ee_m = 0, c_ee_rows = 0;
  cudaError_t ee_reserve(long long n, long long m);
  bool charges_ready() const;
  int launch_ee_pre(long long rows, const nnp::Workspace& w, int& launches);
  void launch_ee_post(int& launches);

  // ML/MM embedding buffers (nnp_mlmm.cu; allocated on first use)
  struct MlmmBufs {
    double *pos = nullptr, *F = nullptr, *sub_pos = nullptr, *sub_F = nullptr, *ld = nullptr, *E = nullptr;
    int32_t *Z = nullptr, *sub_Z = nullptr;
    int64_t* idx = nullptr;
    int* mark = nullptr;   // group membership (device index sets)
    int* h_bad = nullptr;  // pinned: validation bits of the last call
    std::vector<unsigned char> mark_host;
    std::vector<double> ld_host;
    size_t c_pos = 0, c_F = 0, c_sub_pos = 0, c_sub_F = 0, c_ld = 0, c_E = 0, c_Z = 0, c_sub_Z = 0, c_idx = 0,
           c_mark = 0;
  } mm;

  // launch shapes, chosen by the autotuner (NNP_FLAG_AUTOTUNE): blocks-per-SM
  // caps of the persistent neighbour, descriptor and descriptor-backward
  // grids; the descriptor's tiles of row pairs, > 0 drawn from the work
  // queue, < 0 in static order (bwd_tile stays -1: the backward takes one row
  // at a time in static order); nbr_dyn: the neighbour kernel's form, bit 0
  // items from the queue, bit 1 each cell's row groups over two warps
  struct Tune { int nbr = 16, fwd = 8, bwd = 16, fwd_tile = -1, bwd_tile = -1, nbr_dyn = 0; } tune;
  long long tuned_key = -1;
  int autotune(long long n, int B, long long bins, long long rows);

  // stage events (NNP_FLAG_STAGE_EVENTS)
  cudaEvent_t stage_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // force matching: start, forces, tangent descriptors, then per member the
  // end of its network pass and of its weight-gradient jobs
  cudaEvent_t fm_ev[3 + 2 * NNP_MAX_MEMBERS] = {};
  int fm_profiled_members = 0;
  void mark_stage(int k, bool capturing);

  // graph
  cudaGraphExec_t gexec = nullptr;
  long long g_key_n = -1, g_key_bins = -1;
  int g_key_B = -1;
  long long graph_captures = 0;

  // last evaluation
  std::vector<nnp::SysDesc> sys_h;
  long long last_n = 0, last_rows = 0;
  int last_B = 0;
  bool has_state = false;
  long long launches_per_eval = 0;
  int max_nbr_r = 0, max_nbr_a = 0;

  ~nnp_ctx();
  int init_device();
  int fail(int code, const char* fmt, ...);
  int cuda_fail(cudaError_t e, const char* what);
  int ensure_capacity(long long n, int B, long long bins, long long rows);
  nnp::Workspace workspace() const;
  void invalidate_graph();
  int launch_pipeline(long long n, int B, long long bins, long long rows, bool calib = false);
  int prepare(int B, const int64_t* offsets, const double* pos_host, const double* boxes,
              long long& bins, long long& rows);
  int read_flags(int& fl);
  int evaluate(int B, const int64_t* offsets, const double* pos, const int32_t* Z,
               const double* boxes, double* energies, double* forces, bool sync);
  int check_flags();
  bool weights_ready() const;
  int set_weights(int member, int species, const float* const W[4], const float* const b[4]);
  int force_match_grad(const double* v, const double* Fref, double* loss, double* grad);
  int profile_stages(double* out, int n_out);
  int profile_force_match(double* out, int n_out);
};
