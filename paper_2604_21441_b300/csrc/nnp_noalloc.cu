// nnp_noalloc.cu -- nnp_eval_noalloc: one periodic system's energy and forces
// without any device-memory allocation.
//
// Who needs it: a molecular-dynamics engine that reserves the GPU's memory
// for its own pool when it starts.  Once that pool holds the free memory, a
// cudaMalloc in the middle of a run can fail, and it can also stall the
// device while the engine's other streams are busy.  Such a caller creates
// and fills a context once at start-up, then calls this entry point every
// step: it allocates nothing.
//
// How: every per-call scratch buffer of the evaluation (cell bins, sorted
// rows, neighbour lists, descriptors, their gradients, per-atom energies,
// flags, work-queue counters and the small per-call descriptors) is carved
// out of one file-scope
// static device array, g_noalloc_scratch, of fixed size.  The kernels are the
// library's ordinary kernels; only the workspace they are given differs.
// Weights and model constants come from the context.
//
// Host code cannot use the array's name as a device address.  nnp_create
// looks the address up with cudaGetSymbolAddress (its device current) and
// caches it per device (noalloc_prepare).  That lookup also loads this file's
// module, which is when the driver places the array in device memory, and it
// loads the kernels this entry point launches directly; so an MD engine that
// creates its context before it takes the GPU's free memory finds the array
// already in place.  All calls share the array and it keeps the last call's
// contents: the bin counters are cleared at the start of every call, and
// calls that overlap on the GPU (from other streams, contexts or threads)
// race and give wrong results.
#include <cmath>
#include <cstring>
#include <mutex>

#include "nnp_host.h"

using namespace nnp;

namespace {

constexpr long long kNAMaxAtoms = NNP_NOALLOC_MAX_ATOMS;
constexpr int kNACapR = 128;  // radial neighbours per atom
constexpr int kNACapA = 48;   // angular neighbours per atom
constexpr int kNAMaxS = 4;    // species (the scratch array is sized for D <= 384)
constexpr long long kNAMaxRows = kNAMaxAtoms + (long long)kTileRows * kNAMaxS;
constexpr long long kNAMaxCells = 2 * kNAMaxAtoms;  // cell cap per system (>= 27)
constexpr long long kNAMaxBins = kNAMaxS * kNAMaxCells;
constexpr int kNAMaxD = desc_len(kNAMaxS);

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Byte offsets of the sub-arrays inside the scratch array.
constexpr size_t o_bin_count = 0;
constexpr size_t o_bin_start = o_bin_count + al256(sizeof(int) * kNAMaxBins);
constexpr size_t o_bin_len = o_bin_start + al256(sizeof(int) * (kNAMaxBins + 1));
constexpr size_t o_atom_bin = o_bin_len + al256(sizeof(int) * kNAMaxBins);
constexpr size_t o_atom_slot = o_atom_bin + al256(sizeof(int) * kNAMaxAtoms);
constexpr size_t o_atom_off = o_atom_slot + al256(sizeof(int) * kNAMaxAtoms);
constexpr size_t o_atom_cell = o_atom_off + al256(sizeof(float4) * kNAMaxAtoms);
constexpr size_t o_atom_sys = o_atom_cell + al256(sizeof(int) * kNAMaxAtoms);
constexpr size_t o_seg = o_atom_sys + al256(sizeof(int) * kNAMaxAtoms);
constexpr size_t o_row_atom = o_seg + al256(sizeof(int) * (kMaxS + 2));
constexpr size_t o_pos4 = o_row_atom + al256(sizeof(int) * kNAMaxRows);
constexpr size_t o_row_info = o_pos4 + al256(sizeof(float4) * kNAMaxRows);
constexpr size_t o_row_cell = o_row_info + al256(sizeof(int) * kNAMaxRows);
constexpr size_t o_cnt_r = o_row_cell + al256(sizeof(int) * kNAMaxRows);
constexpr size_t o_cnt_a = o_cnt_r + al256(sizeof(int) * kNAMaxRows * kMaxS);
constexpr size_t o_nbr_r = o_cnt_a + al256(sizeof(int) * kNAMaxRows * kMaxS);
constexpr size_t o_G = o_nbr_r + al256(sizeof(int) * kNAMaxRows * kNACapR);
constexpr size_t o_dEdG = o_G + al256(sizeof(float) * kNAMaxRows * kNAMaxD);
constexpr size_t o_Ei = o_dEdG + al256(sizeof(float) * kNAMaxRows * kNAMaxD);
constexpr size_t o_flags = o_Ei + al256(sizeof(float) * kNAMaxRows);
constexpr size_t o_queue = o_flags + al256(sizeof(int) * kNumFlags);
constexpr size_t o_io = o_queue + al256(sizeof(int) * kQueueWords);
constexpr size_t o_sys = o_io + al256(sizeof(EvalIO));
constexpr size_t kScratchBytes = o_sys + al256(sizeof(SysDesc));
static_assert(kScratchBytes <= 8u * 1024u * 1024u, "scratch must stay within 8 MiB");

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int grid_cap(long long items, int per_block, int cap) {
  long long g = (items + per_block - 1) / per_block;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

// The scratch memory of every nnp_eval_noalloc call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// Device address of the scratch array on device `dev` (the current device),
// looked up once and cached.
cudaError_t scratch_base(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

namespace nnp {

// Called by nnp_create with the context's device current: resolves the
// scratch array (which loads its module and places the array in device
// memory) and loads the cell-list kernels that nnp_eval_noalloc launches
// itself.  The other kernels it launches are loaded by the context's own
// set-up (their shared-memory limits are set there).
int noalloc_prepare(nnp_ctx* ctx) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return NNP_OK;  // nnp_eval_noalloc refuses such a device
  unsigned char* base = nullptr;
  e = scratch_base(dev, &base);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  cudaFuncAttributes fa;
  const void* kernels[] = {(const void*)k_bin, (const void*)k_scan, (const void*)k_scatter,
                           (const void*)k_binsort};
  for (const void* k : kernels) {
    e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaFuncGetAttributes");
  }
  return NNP_OK;
}

}  // namespace nnp

extern "C" int nnp_eval_noalloc(nnp_ctx* ctx, int64_t n, const double* pos, const int32_t* Z,
                                const double* box, double* energy, double* forces) {
  if (!ctx) return NNP_ERR_INVALID_ARG;
  if (n <= 0) return ctx->fail(NNP_ERR_INVALID_ARG, "n must be positive");
  if (n > kNAMaxAtoms)
    return ctx->fail(NNP_ERR_CAPACITY, "nnp_eval_noalloc takes at most %d atoms (got %lld)",
                     NNP_NOALLOC_MAX_ATOMS, (long long)n);
  if (!pos || !Z || !energy || !forces || !box)
    return ctx->fail(NNP_ERR_INVALID_ARG, "nnp_eval_noalloc needs pos, Z, energy, forces and a box");
  if (!on_device(pos) || !on_device(Z) || !on_device(energy) || !on_device(forces))
    return ctx->fail(NNP_ERR_INVALID_ARG, "nnp_eval_noalloc needs device pointers for pos, Z, energy, forces");
  if (on_device(box)) return ctx->fail(NNP_ERR_INVALID_ARG, "nnp_eval_noalloc needs the box as a host pointer");
  if (ctx->cfg.precision != NNP_FP32)
    return ctx->fail(NNP_ERR_UNSUPPORTED, "nnp_eval_noalloc supports FP32 contexts only");
  if (ctx->P.S > kNAMaxS)
    return ctx->fail(NNP_ERR_UNSUPPORTED, "nnp_eval_noalloc supports at most %d species", kNAMaxS);
  if (!ctx->weights_ready()) return ctx->fail(NNP_ERR_NO_WEIGHTS, "weights missing for some species");

  // device address of the scratch array (once per device, that device current)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return ctx->fail(NNP_ERR_UNSUPPORTED, "device index %d", dev);
  unsigned char* base = nullptr;  // cached by nnp_create on the context's device
  e = scratch_base(dev, &base);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");

  // one periodic orthorhombic system (same cell rule as nnp_eval)
  SysDesc sd{};
  memset(&sd, 0, sizeof sd);
  const double rc = ctx->cfg.rc_r;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      if (!std::isfinite(box[3 * r + c])) return ctx->fail(NNP_ERR_INVALID_ARG, "non-finite box entry");
      if (r != c && box[3 * r + c] != 0.0)
        return ctx->fail(NNP_ERR_UNSUPPORTED, "triclinic boxes are not supported");
    }
  int nc[3];
  for (int c = 0; c < 3; ++c) {
    const double L = box[4 * c];
    if (!(L > 0.0)) return ctx->fail(NNP_ERR_INVALID_ARG, "box edge %d is %g", c, L);
    if (L < rc) return ctx->fail(NNP_ERR_UNSUPPORTED, "box edge %g is shorter than the radial cutoff %g", L, rc);
    sd.L[c] = L;
    nc[c] = (int)std::floor(L / rc);
    if (nc[c] < 1) nc[c] = 1;
  }
  const long long cap_cells = n * 2 > 27 ? n * 2 : 27;
  while ((long long)nc[0] * nc[1] * nc[2] > cap_cells) {
    const int c = (nc[0] >= nc[1] && nc[0] >= nc[2]) ? 0 : (nc[1] >= nc[2] ? 1 : 2);
    nc[c] = nc[c] * 3 / 4 > 1 ? nc[c] * 3 / 4 : 1;
  }
  for (int c = 0; c < 3; ++c) {
    sd.nc[c] = nc[c];
    sd.ell[c] = sd.L[c] / nc[c];
    sd.inv_L[c] = 1.0 / sd.L[c];
    sd.inv_ell[c] = 1.0 / sd.ell[c];
    sd.ellf[c] = (float)sd.ell[c];
  }
  sd.tric = 0;
  set_cell_steps(sd);
  sd.periodic = 1;
  sd.atom_begin = 0;
  sd.atom_end = n;
  sd.cell_base = 0;
  const long long cells = (long long)nc[0] * nc[1] * nc[2];
  const long long bins = cells * ctx->P.S;
  const long long rows = n + (long long)kTileRows * ctx->P.S;
  if (bins > kNAMaxBins || rows > kNAMaxRows)
    return ctx->fail(NNP_ERR_CAPACITY, "nnp_eval_noalloc: cell grid exceeds its scratch");

  EvalIO io{};
  io.pos = pos;
  io.Z = Z;
  io.forces = forces;
  io.energies = energy;
  io.n_atoms = n;
  io.n_sys = 1;
  io.total_cells = (int)cells;

  Workspace w{};
  w.bin_count = reinterpret_cast<int*>(base + o_bin_count);
  w.bin_start = reinterpret_cast<int*>(base + o_bin_start);
  w.bin_len = reinterpret_cast<int*>(base + o_bin_len);
  w.atom_bin = reinterpret_cast<int*>(base + o_atom_bin);
  w.atom_slot = reinterpret_cast<int*>(base + o_atom_slot);
  w.atom_off = reinterpret_cast<float4*>(base + o_atom_off);
  w.atom_cell = reinterpret_cast<int*>(base + o_atom_cell);
  w.atom_sys = reinterpret_cast<int*>(base + o_atom_sys);
  w.seg = reinterpret_cast<int*>(base + o_seg);
  w.row_atom = reinterpret_cast<int*>(base + o_row_atom);
  w.pos4 = reinterpret_cast<float4*>(base + o_pos4);
  w.row_info = reinterpret_cast<int*>(base + o_row_info);
  w.row_cell = reinterpret_cast<int*>(base + o_row_cell);
  w.cnt_r = reinterpret_cast<int*>(base + o_cnt_r);
  w.cnt_a = reinterpret_cast<int*>(base + o_cnt_a);
  w.nbr_r = reinterpret_cast<int*>(base + o_nbr_r);
  w.G = reinterpret_cast<float*>(base + o_G);
  w.Gh = reinterpret_cast<__nv_bfloat16*>(base + o_G);  // unused: FP32 form writes no BF16 copy
  w.dEdG = reinterpret_cast<float*>(base + o_dEdG);
  w.Ei = reinterpret_cast<float*>(base + o_Ei);
  w.flags = reinterpret_cast<int*>(base + o_flags);
  w.queue = reinterpret_cast<int*>(base + o_queue);
  w.cap_r = kNACapR;
  w.cap_a = kNACapA;
  w.max_rows = kNAMaxRows;
  EvalIO* d_io = reinterpret_cast<EvalIO*>(base + o_io);
  SysDesc* d_sys = reinterpret_cast<SysDesc*>(base + o_sys);

  cudaStream_t st = ctx->stream;
  const DescParams& P = ctx->P;
  const int nsm = ctx->num_sms;
  const int g_atoms = grid_cap(n, 256, nsm * 8);
  const int g_cells = grid_cap(bins / P.S, kNbrThreads / 32, nsm * 16);
  const int g_bins = grid_cap(bins * 32, 256, nsm * 16);
  const int g_tiles = (int)((rows / 64) < nsm ? (rows / 64) : nsm);
  int hflags[kNumFlags];

#define NA_CK(call)                                              \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call);     \
  } while (0)
  // the array keeps the last call's contents: clear what must start at zero
  NA_CK(cudaMemsetAsync(w.bin_count, 0, sizeof(int) * bins, st));
  NA_CK(cudaMemsetAsync(w.flags, 0, sizeof(int) * kNumFlags, st));
  NA_CK(cudaMemsetAsync(w.queue, 0, sizeof(int) * kQueueWords, st));
  NA_CK(cudaMemcpyAsync(d_io, &io, sizeof io, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_sys, &sd, sizeof sd, cudaMemcpyHostToDevice, st));
  k_bin<<<g_atoms, 256, 0, st>>>(d_io, d_sys, ctx->d_zlut, w);
  k_scan<<<1, 1024, sizeof(int) * kScanSmemBins, st>>>(d_io, P.S, w);
  k_scatter<<<g_atoms, 256, 0, st>>>(d_io, w);
  k_binsort<<<g_bins, 256, 0, st>>>(d_io, P.S, 1, w);
  launch_neighbors(g_cells, st, d_io, d_sys, P, w, rows, bins / P.S, nsm);
  launch_aev_fwd(rows, nsm, st, d_sys, P, w, 0);
  for (int m = 0; m < ctx->n_members; ++m)  // ensemble members add up
    launch_mlp_f32(g_tiles > 0 ? g_tiles : 1, st, d_io, P, w, ctx->wf32m[(size_t)m], m > 0 ? 1 : 0);
  launch_aev_bwd(rows, nsm, st, d_io, d_sys, P, w);
  NA_CK(cudaGetLastError());
  NA_CK(cudaMemcpyAsync(hflags, w.flags, sizeof hflags, cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
  if (hflags[kFlagNonFinite]) return ctx->fail(NNP_ERR_INVALID_ARG, "non-finite atom position");
  if (hflags[kFlagBadSpecies])
    return ctx->fail(NNP_ERR_UNKNOWN_SPECIES, "atomic number outside the configured species");
  if (hflags[kFlagOverflowR] || hflags[kFlagOverflowA])
    return ctx->fail(NNP_ERR_CAPACITY,
                     "nnp_eval_noalloc: more than %d radial or %d angular neighbours (%d, %d)",
                     kNACapR, kNACapA, hflags[kFlagMaxNbrR], hflags[kFlagMaxNbrA]);
  return NNP_OK;
}
