// k_pairs.cu -- neighbour lists from a pair list supplied by the caller
// (Methods, "The nnpot Interface in GROMACS": the 2026 interface passes the
// MD engine's own pair list to the model), in place of the cell search.
//
// Input: n_pairs pairs (i, j) with optional Cartesian shifts s, displacement
// d = r_j - r_i + s; every unordered pair (or periodic self-image) once.
// Pairs whose distance is over 1.001 rc_r are dropped at once.  Each
// other pair is placed by its image code: the virtual-cell offset m in
// {-1,0,1}^3 with d = (off_j + m ell) - off_i in the rows' cell-local offsets
// (m from the displacement; a residual that is not a whole number of cell
// lengths, or |m| > 1, marks the pair list invalid).  The keep/drop
// decision then repeats the cell search's own FP32 arithmetic, so a complete
// list yields exactly the lists of the search (up to their order): radial if
// |d|^2 < rc_r^2, angular if also < rc_a^2, both directions.  Buffered lists
// (pairs beyond the cutoff) are fine; a pair listed twice counts twice.
//
//   k_pairs_prep     zero the counts; atom -> row (in atom_slot)
//   k_pairs_count    per (row, neighbour species): angular and radial-only
//   k_pairs_offsets  segment bases, counts clamped to the list capacity,
//                    overflow flags (the host regrows and repeats)
//   k_pairs_fill     entries through atomic cursors (angular part of each
//                    species segment first; order within a part unspecified)
#include "nnp_internal.cuh"

namespace nnp {

__global__ void k_pairs_prep(int S, Workspace ws) {
  const int rows = ws.seg[S];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    for (int s = 0; s < S; ++s) {
      ws.cnt_r[(size_t)r * kMaxS + s] = 0;
      ws.cnt_a[(size_t)r * kMaxS + s] = 0;
    }
    const int a = ws.row_atom[r];
    if (a >= 0) ws.atom_slot[a] = r;
  }
}

namespace {

// One pair: rows, species, image code (-1: invalid, -2: beyond the cutoff) and, per direction
// (0: j in row i's list, 1: i in row j's), the radial and angular decisions.
struct PairGeo {
  int ri, rj, si, sj, code;
  bool radial[2], angular[2];
};

__device__ __forceinline__ PairGeo pair_geo(const EvalIO* __restrict__ io, const SysDesc* __restrict__ sys,
                                            const DescParams& P, const Workspace& ws, long long p) {
  PairGeo g;
  g.code = -1;
  g.radial[0] = g.radial[1] = g.angular[0] = g.angular[1] = false;
  const long long n = io->n_atoms;
  const int i = io->pairs[2 * p], j = io->pairs[2 * p + 1];
  if (i < 0 || i >= n || j < 0 || j >= n) return g;
  // FP32 throughout (this part's FP64 rate is a small fraction of its FP32
  // rate): at 100 A the displacement is good to ~1e-5 A, far inside the
  // prefilter's margin and the image test's tolerance
  float d[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    d[c] = ((float)io->pos[3 * j + c] - (float)io->pos[3 * i + c]) + (io->shifts ? (float)io->shifts[3 * p + c] : 0.f);
  // pairs clearly beyond the cutoff (buffered lists) are dropped before any image test
  const float rcap = 1.001f * P.rc_r;
  if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] >= rcap * rcap) {
    g.code = -2;
    return g;
  }
  g.ri = ws.atom_slot[i];
  g.rj = ws.atom_slot[j];
  const float4 pi = ws.pos4[g.ri], pj = ws.pos4[g.rj];
  g.si = pos4_species(pi);
  g.sj = pos4_species(pj);
  const SysDesc& sd = sys[ws.row_info[g.ri]];
  // the image in cell steps: m = (d - (off_j - off_i)) cv^-1
  const float x[3] = {d[0] - (pj.x - pi.x), d[1] - (pj.y - pi.y), d[2] - (pj.z - pi.z)};
  int m[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float q = x[0] * sd.cvinv[c] + x[1] * sd.cvinv[3 + c] + x[2] * sd.cvinv[6 + c];
    m[c] = __float2int_rn(q);
    if (m[c] < -1 || m[c] > 1 || fabsf(q - (float)m[c]) > 1e-3f) return g;
  }
  g.code = (m[0] + 1) * 9 + (m[1] + 1) * 3 + (m[2] + 1);
  // the cell search's arithmetic, per direction: candidate = off + m ell
  // (FP32), then its distance to the row's own offset
  const float rcr2 = P.rc_r * P.rc_r, rca2 = P.rc_a * P.rc_a;
  const bool self = g.ri == g.rj && g.code == 13;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const float4 a = side ? pj : pi, b = side ? pi : pj;
    const int sg = side ? -1 : 1;
    const float3 v = cell_shift(sg * m[0], sg * m[1], sg * m[2], sd);
    const float cx = b.x + v.x, cy = b.y + v.y, cz = b.z + v.z;
    const float dx = cx - a.x, dy = cy - a.y, dz = cz - a.z;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));  // the search's rounding order
    g.radial[side] = r2 < rcr2 && !self;
    g.angular[side] = g.radial[side] && r2 < rca2;
  }
  return g;
}

}  // namespace

// Lanes that add to the same (row, species, kind) counter are grouped by
// __match_any_sync and one lane adds for the group: pair lists are usually
// ordered by their first atom, so a warp would otherwise queue up to 32
// atomics on one address.  The loops step whole warps, so every lane takes
// part in the match.
namespace {
__device__ __forceinline__ unsigned key_of(int row, int s, bool ang) {
  return ((unsigned)row << 4) | ((unsigned)s << 1) | (ang ? 0u : 1u);  // s < 8, rows < 2^28
}
}  // namespace

__global__ void k_pairs_count(const EvalIO* __restrict__ io, const SysDesc* __restrict__ sys, DescParams P,
                              Workspace ws) {
  const long long np = io->n_pairs;
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); p0 < np; p0 += stride) {
    const long long p = p0 + lane;
    PairGeo g;
    g.code = -2;
    if (p < np) g = pair_geo(io, sys, P, ws, p);
    if (g.code == -1) atomicOr(&ws.flags[kFlagBadPair], 1);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const bool act = g.code >= 0 && g.radial[side];
      const int r = side ? g.rj : g.ri, so = side ? g.si : g.sj;
      const unsigned key = act ? key_of(r, so, g.angular[side]) : 0xffffffffu;
      const unsigned grp = __match_any_sync(0xffffffffu, key);
      // radial-only counts in cnt_r until k_pairs_offsets
      if (act && lane == __ffs(grp) - 1)
        atomicAdd(&(g.angular[side] ? ws.cnt_a : ws.cnt_r)[(size_t)r * kMaxS + so], __popc(grp));
    }
  }
}

__global__ void k_pairs_offsets(const EvalIO* __restrict__ io, int S, Workspace ws, int* __restrict__ cur) {
  const int rows = ws.seg[S], cap = ws.cap_r;
  int mx_r = 0, mx_a = 0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    int nr = 0, tot = 0, tang = 0;
    for (int s = 0; s < S; ++s) {
      const int a = ws.cnt_a[(size_t)r * kMaxS + s], ro = ws.cnt_r[(size_t)r * kMaxS + s];
      const int keep = max(0, min(a + ro, cap - nr));  // counts clamped to what the list holds
      cur[(size_t)r * 2 * kMaxS + 2 * s] = nr;          // angular cursor
      cur[(size_t)r * 2 * kMaxS + 2 * s + 1] = nr + a;  // radial-only cursor
      ws.cnt_r[(size_t)r * kMaxS + s] = keep;
      ws.cnt_a[(size_t)r * kMaxS + s] = min(a, keep);
      nr += keep;
      tot += a + ro;
      tang += a;
    }
    mx_r = max(mx_r, tot);
    mx_a = max(mx_a, tang);
  }
  if (mx_r | mx_a) {
    atomicMax(&ws.flags[kFlagMaxNbrR], mx_r);
    atomicMax(&ws.flags[kFlagMaxNbrA], mx_a);
    if (mx_r > ws.cap_r) atomicOr(&ws.flags[kFlagOverflowR], 1);
    if (mx_a > ws.cap_a) atomicOr(&ws.flags[kFlagOverflowA], 1);
  }
}

__global__ void k_pairs_fill(const EvalIO* __restrict__ io, const SysDesc* __restrict__ sys, DescParams P,
                             Workspace ws, int* __restrict__ cur) {
  const long long np = io->n_pairs;
  const int cap = ws.cap_r, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); p0 < np; p0 += stride) {
    const long long p = p0 + lane;
    PairGeo g;
    g.code = -2;
    if (p < np) g = pair_geo(io, sys, P, ws, p);
    // (row, its neighbour's row, neighbour species, code), per direction
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const bool act = g.code >= 0 && g.radial[side];
      const bool ang = g.angular[side];
      const int r = side ? g.rj : g.ri, o = side ? g.ri : g.rj, so = side ? g.si : g.sj;
      const unsigned key = act ? key_of(r, so, ang) : 0xffffffffu;
      const unsigned grp = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(grp) - 1;
      int q0 = 0;
      if (act && lane == leader) q0 = atomicAdd(&cur[(size_t)r * 2 * kMaxS + 2 * so + (ang ? 0 : 1)], __popc(grp));
      q0 = __shfl_sync(0xffffffffu, q0, leader);
      if (!act) continue;
      const int q = q0 + __popc(grp & lt);
      int base = 0;
      for (int s = 0; s < so; ++s) base += ws.cnt_r[(size_t)r * kMaxS + s];
      const int lim = base + (ang ? ws.cnt_a[(size_t)r * kMaxS + so] : ws.cnt_r[(size_t)r * kMaxS + so]);
      if (q < lim && q < cap) ws.nbr_r[(size_t)r * cap + q] = pack_nbr(o, side ? 26 - g.code : g.code);
    }
  }
}

}  // namespace nnp
