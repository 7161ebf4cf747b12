// nnp_internal.cuh -- device-side layouts and helpers shared by the libnnp
// kernels (private to the library).
//
// Data layout in HBM (one evaluation, B systems, N atoms):
//   * rows: atoms sorted species-major, then by system, then by cell
//     (ascending input index inside a cell).  Each species segment starts on
//     a multiple of kTileRows so that every network tile holds one species.
//     Padding rows have row_atom = -1 and an all-zero descriptor.
//   * pos4[row] = (x, y, z offset of the atom from its cell's lower corner in
//     FP32, bits(orig << 3 | species)): displacements are formed as
//     (off_j - off_i) + m * ell with m in {-1, 0, 1}^3, so FP32 rounding does
//     not grow with the box edge.
//   * neighbour entries: row index j (27 bits) | image code (5 bits), code =
//     (mx+1)*9 + (my+1)*3 + (mz+1).  One list per row, grouped by neighbour
//     species; inside a species segment the entries within the angular
//     cutoff come first (cnt_a of them), then the radial-only ones (cnt_r
//     counts the whole segment).
//   * G / dEdG: row-major [rows][D] FP32 (plus a BF16 copy for tensor cores).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace nnp {

constexpr int kNRad = 16;      // radial shifts
constexpr int kNAngR = 4;      // angular radial shifts
constexpr int kNAngZ = 8;      // angular sectors
constexpr int kNAng = kNAngR * kNAngZ;  // 32 features per species pair
constexpr int kH1 = 160, kH2 = 128, kH3 = 96;
constexpr int kMaxS = 8;       // species supported by the kernels (stride of the per-row counts)
constexpr int kTileRows = 128; // species segments are padded to this
constexpr int kMaxCapA = 64;     // largest angular-neighbour capacity (staged per row)
constexpr int kMaxCapR = 512;    // largest radial-neighbour capacity (gathered per row)
constexpr int kScanSmemBins = 49152;  // k_scan stages up to this many bins in shared memory (192 KB)
constexpr int kScanSmemBinsSmall = 16384;  // the same for k_cells_small (64 KB, also its sort buffers)
constexpr int kNbrThreads = 128;  // k_neighbors: warp per cell, lane per row
constexpr int kNbrWin = 512;      // neighbourhood atoms one warp stages per window
constexpr int kNbrWinSmall = 1024;          // the same for small systems (at most kNbrRowsSmall rows)
constexpr int kNbrWinTiny = 2048;           // one-cell systems (27 images of the cell)
constexpr long long kNbrRowsSmall = 8192;
constexpr long long kCellsRowsSmall = 1536;  // up to this many rows the binning runs in one block
constexpr int kNbrChunkStride = 36;       // floats per chunk in shared memory (bank spread)
constexpr size_t kG1TileBytes = 3 * 128 * 128;  // one 128-row g1 tile (K = 160 in three swizzled slabs), BF16
constexpr int kMaxD = kNRad * kMaxS + kNAng * kMaxS * (kMaxS + 1) / 2;  // 1280
__host__ __device__ constexpr int desc_len(int S) { return kNRad * S + kNAng * S * (S + 1) / 2; }

// switch cases over the species count, CALL(s) with s a constant 1..kMaxS
#define NNP_SPECIES_CASES(CALL)                                                      \
  case 1: CALL(1); break;                                                            \
  case 2: CALL(2); break;                                                            \
  case 3: CALL(3); break;                                                            \
  case 4: CALL(4); break;                                                            \
  case 5: CALL(5); break;                                                            \
  case 6: CALL(6); break;                                                            \
  case 7: CALL(7); break;                                                            \
  default: CALL(8); break;


// Error flag words (device): set by kernels, read by the host after sync.
enum FlagWord {
  kFlagBadSpecies = 0,
  kFlagNonFinite = 1,
  kFlagOverflowR = 2,   // radial list overflow
  kFlagOverflowA = 3,   // angular list overflow
  kFlagMaxNbrR = 4,     // max radial count seen (atomicMax)
  kFlagMaxNbrA = 5,
  kFlagBinOverflow = 6, // a bin held more than the per-bin sort capacity
  kFlagTimeout = 7,
  kFlagBadPair = 8,     // a caller's pair: index out of range or shift not a whole image
  kFlagChecked = 9,     // bounds-checked build: an index read from device data was out of range
  kFlagCheckedLine = 10,  // its source line and value (the first one recorded)
  kFlagCheckedValue = 11,
  kFlagFp8Uncal = 12,   // FP8: a tile's species has no calibrated activation range yet
  kNumFlags = 13
};

// Descriptor and network constants, passed by value to kernels.
struct DescParams {
  int S;              // species
  int D;              // descriptor length
  int zeta_sq;        // zeta = 2^zeta_sq
  float rc_r, eta_r, rc_a, eta_a;
  float shf_r[kNRad];
  float shf_a[kNAngR];
  float hcos_z[kNAngZ], hsin_z[kNAngZ];  // cos(theta_z)/2, sin(theta_z)/2
  float celu_alpha;
  // evenly spaced radial shifts R_m = R_0 + m dR (rad_even = 1): the BF16
  // and FP8 forms' descriptor kernel takes exp(-eta_r (r - R_m)^2) from the
  // anchors m = 4 and 12 by the ratio of neighbouring terms,
  //   e_{A+-d} = e_{A+-(d-1)} * exp(+-2 eta_r dR (r - R_A)) * exp(-eta_r dR^2 (2d - 1)),
  // rad_gk = 2 eta_r dR log2(e), rad_c[d - 1] = exp(-eta_r dR^2 (2d - 1))
  int rad_even;
  float rad_gk;
  float rad_c[4];
};

// One periodic system.  Filled on the host, copied to the device per eval.
// Orthorhombic boxes and isolated systems use the edge form (L, ell); a
// triclinic box (tric = 1) wraps through fractional coordinates s = r Binv
// with B's rows the cell vectors a, b, c.  In both forms cell (k0, k1, k2)
// has its corner at sum_d k_d cv_d and the image shift of virtual-cell offset
// m is sum_d m_d cv_d (cv = B / nc row-wise; diagonal for the edge form).
struct SysDesc {
  double L[3];      // edges (isolated systems: padded bounding box)
  double ell[3];    // cell edges L / nc
  double inv_L[3], inv_ell[3];  // reciprocals (the wrap multiplies: FP64 division is slow)
  double origin[3]; // subtracted before wrapping (isolated systems)
  double B[9], Binv[9];  // triclinic: cell vectors (rows) and the inverse, s_d = sum_c r_c Binv[c][d]
  float ellf[3];
  float cv[9];      // cell steps: rows cv_d = B_d / nc_d
  float cvinv[9];   // inverse of cv (rows), for image codes of given displacements
  int nc[3];
  int cell_base;    // first global cell of this system
  int periodic;
  int tric;
  long long atom_begin, atom_end;
};

// Image shift of virtual-cell offset (m0, m1, m2): sum_d m_d cv_d, in one
// fixed FP32 order shared by every kernel (exactly m_d ell_d for the edge form).
__device__ __forceinline__ float3 cell_shift(int m0, int m1, int m2, const SysDesc& sd) {
  float3 v;
  v.x = fmaf((float)m2, sd.cv[6], fmaf((float)m1, sd.cv[3], (float)m0 * sd.cv[0]));
  v.y = fmaf((float)m2, sd.cv[7], fmaf((float)m1, sd.cv[4], (float)m0 * sd.cv[1]));
  v.z = fmaf((float)m2, sd.cv[8], fmaf((float)m1, sd.cv[5], (float)m0 * sd.cv[2]));
  return v;
}

// Per-evaluation IO descriptor (device memory, refreshed before each launch
// so that captured graphs do not depend on caller pointers).
struct EvalIO {
  const double* pos;   // n x 3
  const int* Z;        // n
  double* forces;      // n x 3 (zeroed by the bin kernel)
  double* energies;    // B (zeroed by the bin kernel)
  long long n_atoms;
  int n_sys;
  int total_cells;     // sum of cells over systems
  const int* pairs;     // caller's pair list (n_pairs x 2), or null: the cell search
  const double* shifts; // n_pairs x 3, or null
  long long n_pairs;
};

// Electrostatic embedding parameters and buffers of one evaluation (device
// copy read by the embedding kernels; see nnp_ee.cu).
struct EeIO {
  const double* mm_pos;   // n_mm x 3
  const double* mm_q;     // n_mm
  long long n_mm;
  double Q;               // total charge of the ML atoms
  int S;                  // species (rows = seg[S])
  int periodic;           // orthorhombic minimum image
  float Lhi[3], Llo[3];    // box edges as FP32 hi + lo
  double L[3], invL[3];    // and in FP64 (coordinates are wrapped into [0, L))
  float4 *mm_hi, *mm_lo;  // MM coordinates as FP32 hi + lo, charge in mm_hi.w
  float4 *ml_hi, *ml_lo;  // ML coordinates, input order
  double* V;              // n: potential of the MM charges at each ML atom (eV / e)
  double* field;          // n x 3: -grad V
  float* q_rows;          // [rows] raw charges from the charge network
  float* dqdG;            // [rows][D] their descriptor gradients
  double* q_atom;         // n: raw charges in input order
  double* q_out;          // n: charges shifted to the total charge (output)
  double* mm_forces;      // n_mm x 3 (output)
  double* sums;           // [0] scratch, [1] sum of V, [2] sum of raw charges
};

// Device workspace (all capacity-sized).
struct Workspace {
  // binning
  int* bin_count;   // [S * max_cells]
  int* bin_start;   // [S * max_cells + 1]
  int* bin_len;     // [S * max_cells]
  int* atom_bin;    // [max_atoms]
  int* atom_slot;   // [max_atoms]
  float4* atom_off; // [max_atoms]  (offsets, bits(orig<<3|s))
  int* atom_cell;   // [max_atoms]  packed local cell
  int* atom_sys;    // [max_atoms]  system index
  int* seg;         // [kMaxS + 2]: species segment starts (rows), seg[S] = rows
  // rows
  int* row_atom;    // [max_rows]
  float4* pos4;     // [max_rows]
  int* row_info;    // [max_rows]  system index (bits 0..19) ; unused upper
  int* row_cell;    // [max_rows]  local cell (cx | cy << 10 | cz << 20)
  int* cnt_r;       // [max_rows * kMaxS]
  int* cnt_a;       // [max_rows * kMaxS]
  int* nbr_r;       // [max_rows * cap_r]: per neighbour species, angular entries first
  float* G;         // [max_rows * D]
  __nv_bfloat16* Gh;  // [max_rows * D]
  float* dEdG;      // [max_rows * D]
  float* Ei;        // [max_rows]
  int* flags;       // [kNumFlags]
  int* q8;          // FP8 form, [kMaxS * 8] per species: calibrated |max| of G, h1, h2 as
                    // float bits at [0, 3) (raised by atomicMax); the rest unused
  int* queue;       // [kQueueWords] work-queue counters (zero between launches)
  int cap_r;        // radial list capacity per row
  int cap_a;        // angular neighbours per row that the descriptor kernels stage
  long long max_rows;
};

// Work distribution of the persistent kernels.  Static: warp w of the launch
// takes items w, w + W, w + 2W, ... (W warps).  Dynamic: warp w takes item w
// first, then the items after the first W from a queue, one atomic add each,
// requested one item ahead once the warp has finished its first (so the
// requests do not all arrive at the start of the launch).  Each stage has a
// pair of counters (items handed out, warps done); the last warp of a
// dynamic launch to finish puts both back to zero for the next launch.
enum QueueSlot { kQNbr = 0, kQFwd = 2, kQNet = 4, kQueueWords = 8 };

// Bounds-checked build (compiled with -DNNP_CHECKED): an index read from
// device data (a neighbour-list entry, a bin, a slot, a species) is checked
// before it addresses memory.  A bad one raises kFlagChecked, records the
// first source line and value, and the access is skipped; the host then
// returns NNP_ERR_BOUNDS.  In the ordinary build the checks are constant true.
__device__ __forceinline__ bool checked_in(long long i, long long n, int* flags, int line) {
  if (i >= 0 && i < n) return true;
  if (atomicOr(&flags[kFlagChecked], 1) == 0) {
    flags[kFlagCheckedLine] = line;
    flags[kFlagCheckedValue] = (int)i;
  }
  return false;
}
#ifdef NNP_CHECKED
#define NNP_IN(i, n, flags) ::nnp::checked_in((long long)(i), (long long)(n), (flags), __LINE__)
#else
#define NNP_IN(i, n, flags) true
#endif

struct WorkQueue {
  int* q;
  int base;       // warps of the launch
  int cur;        // the warp's current item (static order)
  int req;        // lane 0: the counter value requested ahead
  bool pending;   // a request is in flight (warp-uniform)
  bool dyn;
  __device__ __forceinline__ WorkQueue(int* counters, bool dynamic)
      : q(counters), base((int)(gridDim.x * (blockDim.x >> 5))), cur(0), req(0), pending(false),
        dyn(dynamic) {}
  // the warp's first item
  __device__ __forceinline__ int first() {
    cur = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    return cur;
  }
  // the next item after the one just finished
  __device__ __forceinline__ int next(int lane) {
    if (!dyn) return cur += base;
    if (!pending && lane == 0) req = atomicAdd(q, 1);
    const int it = __shfl_sync(0xffffffffu, req, 0);
    if (lane == 0) req = atomicAdd(q, 1);  // one ahead
    pending = true;
    return base + it;
  }
};

// every warp of a dynamic launch calls this once, after its last request
__device__ __forceinline__ void queue_warp_done(const WorkQueue& wq, int lane) {
  int* q = wq.q;
  if (wq.dyn && lane == 0) {
    __threadfence();
    const int total = (int)(gridDim.x * (blockDim.x >> 5));
    if (atomicAdd(q + 1, 1) == total - 1) {
      atomicExch(q, 0);
      atomicExch(q + 1, 0);
    }
  }
}

// FP32 network weights per species: W_l row-major (fan_in x fan_out) and the
// transposed copies W_l^T used by the backward pass.
struct MlpF32Weights {
  const float* W[kMaxS][4];
  const float* WT[kMaxS][3];  // W1^T, W2^T, W3^T
  const float* b[kMaxS][4];
};

// One block of the force-matching weight-gradient reduction: a 32 x 32 tile
// (i0, o0) of layer l's gradient (l = 4: the output weights), over rows
// [r0, r1) of one species; w_off / b_off index the packed gradient;
// scale multiplies the job's sums (1/M for an ensemble's output weights,
// which are stored divided by M).
struct FmJob {
  int l, i0, o0, r0, r1;
  float scale;
  long long w_off, b_off;
};

// --------------------------------------------------------------------------
// small device helpers

__device__ __forceinline__ int warp_id_global() {
  return (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}

__device__ __forceinline__ float3 image_shift(int code, const float ell[3]) {
  int mx = code / 9 - 1, my = (code / 3) % 3 - 1, mz = code % 3 - 1;
  return make_float3(mx * ell[0], my * ell[1], mz * ell[2]);
}

__device__ __forceinline__ int nbr_row(int e) { return e & 0x07FFFFFF; }
__device__ __forceinline__ int nbr_code(int e) { return (int)((unsigned)e >> 27); }
// packed FP32 pair (fma/mul.rn.f32x2: one instruction for two lanes of arithmetic)
struct f2 {
  unsigned long long v;
};
__device__ __forceinline__ f2 f2_make(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 f2_split(f2 x) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(x.v));
  return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ int pack_nbr(int row, int code) {
  return (int)((unsigned)row | ((unsigned)code << 27));
}

__device__ __forceinline__ int pos4_species(float4 p) {
  return __float_as_int(p.w) & 7;
}
__device__ __forceinline__ int pos4_orig(float4 p) {
  return (int)((unsigned)__float_as_int(p.w) >> 3);
}

// cosine cutoff and its derivative (accurate cospi/sinpi)
__device__ __forceinline__ float cutoff_fc(float r, float rc) {
  return r < rc ? 0.5f * cospif(r / rc) + 0.5f : 0.0f;
}
__device__ __forceinline__ float cutoff_dfc(float r, float rc) {
  return r < rc ? -0.5f * (3.14159265358979f / rc) * sinpif(r / rc) : 0.0f;
}

// Reduce-scatter of V register values over the warp: afterwards lane l
// holds the warp sum of value (l * V / 32) for V = 32 (V = 16: lanes 2k and
// 2k+1 both hold value k).
template <int V>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[V], int lane) {
  static_assert(V == 32 || V == 16, "V must be 16 or 32");
#pragma unroll
  for (int w = V / 2, bit = 16; w >= 1; w >>= 1, bit >>= 1) {
    const bool upper = (lane & bit) != 0;
#pragma unroll
    for (int k = 0; k < w; ++k) {
      float keep = upper ? v[k + w] : v[k];
      float send = upper ? v[k] : v[k + w];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
  float r = v[0];
  if (V == 16) r += __shfl_xor_sync(0xffffffffu, r, 1);
  return r;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// BF16 copy of G for the tensor-core network: each 128-row tile is stored as
// K-major slabs of 64 features (128 bytes per row), 16-byte chunks swizzled
// by (chunk ^ (row & 7)) -- the operand layout tcgen05.mma reads with
// 128-byte swizzling.  Byte offset of feature f of a row:
__host__ __device__ __forceinline__ size_t gh_tile_bytes(int D) {
  return (size_t)((D + 63) / 64) * 128 * 128;
}
__device__ __forceinline__ size_t gh_offset(int row, int f, int D) {
  const int r = row & 127;
  return (size_t)(row >> 7) * gh_tile_bytes(D) + (size_t)(f >> 6) * (128 * 128) + (size_t)r * 128 +
         (size_t)((((f >> 3) & 7) ^ (r & 7)) << 4) + (size_t)(f & 7) * 2;
}

// FP8 (E4M3) copy of G for the FP8 form: the same tiling with 128 one-byte
// features per slab, 16-byte chunks of 16 features swizzled the same way.
__host__ __device__ __forceinline__ size_t gh8_tile_bytes(int D) {
  return (size_t)((D + 127) / 128) * 128 * 128;
}
__device__ __forceinline__ size_t gh8_offset(int row, int f, int D) {
  const int r = row & 127;
  return (size_t)(row >> 7) * gh8_tile_bytes(D) + (size_t)(f >> 7) * (128 * 128) + (size_t)r * 128 +
         (size_t)((((f >> 4) & 7) ^ (r & 7)) << 4) + (size_t)(f & 15);
}

// What the descriptor kernel writes: FP32 G, or the BF16 / FP8 tile copy.
enum GMode { kGFp32 = 0, kGBf16 = 1, kGFp8 = 2 };

// Largest finite E4M3 magnitude; a per-layer scale s = amax / kE4M3Max maps
// the calibrated range onto the format's.
constexpr float kE4M3Max = 448.f;
__device__ __forceinline__ float fp8_step(int amax_bits) {
  const float a = __int_as_float(amax_bits);
  return a > 0.f ? a / kE4M3Max : 1.f;
}

__device__ __forceinline__ int pair_block(int S, int s1, int s2) {
  // row-major upper triangle index of (s1 <= s2)
  return s1 * S - (s1 * (s1 - 1)) / 2 + (s2 - s1);
}

}  // namespace nnp
