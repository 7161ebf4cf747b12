// k_cells.cu -- periodic wrap, cell binning, species-major counting sort and
// neighbour lists (the pair search of the descriptor: every neighbour image
// within the radial cutoff, strict r < rc).
//
// Pipeline (one launch each, grid-stride, sizes read from device memory so
// that a captured CUDA graph stays valid while boxes change):
//   k_bin      atom -> (species, system, cell) bin and a slot in that bin
//   k_scan     bin counts -> row starts; species segments padded to 128 rows
//   k_scatter  atom -> row (slot order, not yet deterministic)
//   k_binsort  order each bin by input index; write the row arrays
//   k_neighbors  warp per cell: the 27-cell neighbourhood staged in shared
//                memory, rows in groups with 2-32 lanes per row; lists
//                grouped by neighbour species, angular entries first
#include "nnp_internal.cuh"

namespace nnp {

// The four binning steps are device functions over (first thread, thread
// stride), so that small systems run them in one block (k_cells_small) and
// large ones as four grid-wide kernels.
//
// stage (k_bin; nullptr in k_cells_small): 48 double2 of shared memory per
// warp.  With it, a warp whose 32 atoms are all present reads their 768 bytes
// of positions as 48 aligned 16-byte pieces and redistributes them through
// shared memory: whole 128-byte requests, which matters most when the
// positions are page-locked host memory read over PCIe.
__device__ __forceinline__ void bin_atoms(const EvalIO* __restrict__ io, const SysDesc* __restrict__ sys,
                                          const signed char* __restrict__ zlut, const Workspace& ws,
                                          long long tid0, long long stride, double2* stage) {
  const long long n = io->n_atoms;
  const int TC = io->total_cells;
  const int nsys = io->n_sys;
  const int lane = threadIdx.x & 31;
  const bool vec = stage != nullptr && (reinterpret_cast<uintptr_t>(io->pos) & 15) == 0;
  for (long long q = tid0; q < nsys; q += stride) io->energies[q] = 0.0;
  // the lanes of a warp go through the loop together (stride is a multiple of 32)
  for (long long a = tid0; a - lane < n; a += stride) {
    double p[3];
    if (vec && a - lane + 32 <= n) {
      const double2* src = reinterpret_cast<const double2*>(io->pos + 3 * (a - lane));
      const double2 c0 = src[lane];
      const double2 c1 = lane < 16 ? src[32 + lane] : make_double2(0.0, 0.0);
      stage[lane] = c0;
      if (lane < 16) stage[32 + lane] = c1;
      __syncwarp();
      const double* sp3 = reinterpret_cast<const double*>(stage) + 3 * lane;
      p[0] = sp3[0];
      p[1] = sp3[1];
      p[2] = sp3[2];
      __syncwarp();  // the stage is rewritten in the next iteration
    } else if (a < n) {
      p[0] = io->pos[3 * a];
      p[1] = io->pos[3 * a + 1];
      p[2] = io->pos[3 * a + 2];
    }
    if (a >= n) continue;
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (sys[mid].atom_begin <= a) lo = mid; else hi = mid - 1;
    }
    const SysDesc& sd = sys[lo];
    const bool finite = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]);
    if (!finite) {
      atomicOr(&ws.flags[kFlagNonFinite], 1);
      p[0] = p[1] = p[2] = 0.0;
    }
    const int z = io->Z[a];
    int s = (z >= 0 && z < 128) ? (int)zlut[z] : -1;
    if (s < 0) {
      atomicOr(&ws.flags[kFlagBadSpecies], 1);
      s = 0;
    }
    int k[3];
    float off[3];
    if (sd.tric) {
      // fractional coordinates, wrapped into [0, 1); the offset from the
      // cell's corner is the fractional remainder times the cell steps
      double f[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double t = p[0] * sd.Binv[d] + p[1] * sd.Binv[3 + d] + p[2] * sd.Binv[6 + d];
        t -= floor(t);
        if (t >= 1.0) t -= 1.0;
        if (t < 0.0) t = 0.0;
        const double u = t * sd.nc[d];
        int kk = (int)floor(u);
        kk = kk < 0 ? 0 : (kk >= sd.nc[d] ? sd.nc[d] - 1 : kk);
        k[d] = kk;
        f[d] = (u - kk) / sd.nc[d];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) off[c] = (float)(f[0] * sd.B[c] + f[1] * sd.B[3 + c] + f[2] * sd.B[6 + c]);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double x = p[c] - sd.origin[c];
        if (sd.periodic) {
          x -= sd.L[c] * floor(x * sd.inv_L[c]);
          if (x >= sd.L[c]) x -= sd.L[c];
          if (x < 0.0) x = 0.0;
        }
        int kk = (int)floor(x * sd.inv_ell[c]);
        kk = kk < 0 ? 0 : (kk >= sd.nc[c] ? sd.nc[c] - 1 : kk);
        k[c] = kk;
        off[c] = (float)(x - kk * sd.ell[c]);
      }
    }
    const int cell = (k[0] * sd.nc[1] + k[1]) * sd.nc[2] + k[2];
    const int bin = s * TC + sd.cell_base + cell;
    ws.atom_slot[a] = atomicAdd(&ws.bin_count[bin], 1);
    ws.atom_bin[a] = bin;
    ws.atom_off[a] = make_float4(off[0], off[1], off[2],
                                 __int_as_float((int)(((unsigned)a << 3) | (unsigned)s)));
    ws.atom_cell[a] = k[0] | (k[1] << 10) | (k[2] << 20);
    ws.atom_sys[a] = lo;
    io->forces[3 * a] = 0.0;  // the descriptor backward adds the forces here in FP64
    io->forces[3 * a + 1] = 0.0;
    io->forces[3 * a + 2] = 0.0;
  }
}

__global__ void k_bin(const EvalIO* __restrict__ io, const SysDesc* __restrict__ sys,
                      const signed char* __restrict__ zlut, Workspace ws) {
  __shared__ double2 s_pos[8][48];  // blocks of 256 threads
  bin_atoms(io, sys, zlut, ws, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x,
            s_pos[(threadIdx.x >> 5) & 7]);
}

// One block of 1024 threads.  bin_start[b] = first row of bin b, with each
// species segment starting on a multiple of kTileRows; bin_len keeps counts.
__device__ __forceinline__ void scan_bins(const EvalIO* __restrict__ io, int S, const Workspace& ws,
                                          int* s_bins /* [cap_bins] shared */, int cap_bins) {
  constexpr int kReg = 16;  // bins per thread held in registers (up to 16,384 bins)
  __shared__ int warp_tot[32];
  __shared__ long long seg_s[kMaxS + 2];
  __shared__ int raw_at_species[kMaxS + 1];
  const int nb = S * io->total_cells;
  const int TC = io->total_cells;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int chunk = (nb + 1023) / 1024;
  const int b0 = t * chunk, b1 = min(nb, b0 + chunk);
  const bool in_smem = nb <= cap_bins;
  const bool in_reg = nb <= 1024 * kReg;  // else (up to kScanSmemBins) the ranges are read from shared memory
  // coalesced loads into shared memory (and bin_len), then each thread scans
  // its contiguous range from there
  if (in_smem) {
    // eight independent loads in flight per thread before their stores
    // (a load after each store would wait a full round trip per bin)
    for (int bb = t; bb < nb; bb += 8 * 1024) {
      int c[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) c[i] = bb + i * 1024 < nb ? ws.bin_count[bb + i * 1024] : 0;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (bb + i * 1024 < nb) {
          s_bins[bb + i * 1024] = c[i];
          ws.bin_len[bb + i * 1024] = c[i];
        }
    }
    __syncthreads();
  }
  int cnt[kReg];
  int sum = 0;
  if (in_reg) {
#pragma unroll
    for (int i = 0; i < kReg; ++i) cnt[i] = (b0 + i < b1) ? s_bins[b0 + i] : 0;
#pragma unroll
    for (int i = 0; i < kReg; ++i) sum += cnt[i];
  } else if (in_smem) {
    for (int b = b0; b < b1; ++b) sum += s_bins[b];
  } else {
    for (int b = b0; b < b1; ++b) sum += ws.bin_count[b];
  }
  // block exclusive scan of per-thread sums
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int v = warp_tot[lane];
    int iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, iv, o);
      if (lane >= o) iv += y;
    }
    warp_tot[lane] = iv - v;  // exclusive warp offsets
  }
  __syncthreads();
  const int run0 = warp_tot[wid] + incl - sum;  // raw prefix (no padding yet) of bin b0
  {
    // bins are species-major: species sp starts at bin sp * TC (no divisions per bin)
    int run = run0;
    int sp = TC > 0 ? b0 / TC : 0, sp_start = sp * TC;
    if (in_reg) {
#pragma unroll
      for (int i = 0; i < kReg; ++i) {
        const int b = b0 + i;
        if (b < b1) {
          if (b == sp_start + TC) {
            ++sp;
            sp_start += TC;
          }
          if (b == sp_start) raw_at_species[sp] = run;
          s_bins[b] = run;  // raw start
        }
        run += cnt[i];
      }
    } else if (in_smem) {
      for (int b = b0; b < b1; ++b) {
        if (b == sp_start + TC) {
          ++sp;
          sp_start += TC;
        }
        if (b == sp_start) raw_at_species[sp] = run;
        const int c = s_bins[b];
        s_bins[b] = run;  // raw start
        run += c;
      }
    } else {
      for (int b = b0; b < b1; ++b) {
        if (b == sp_start + TC) {
          ++sp;
          sp_start += TC;
        }
        if (b == sp_start) raw_at_species[sp] = run;
        run += ws.bin_count[b];
      }
    }
    if (b1 == nb && b0 < b1) raw_at_species[S] = run;
  }
  if (nb == 0 && t == 0) raw_at_species[S] = 0;
  __syncthreads();
  if (t == 0) {
    long long start = 0;
    for (int s = 0; s < S; ++s) {
      seg_s[s] = start;
      const int c = raw_at_species[s + 1] - raw_at_species[s];
      start = ((start + c + kTileRows - 1) / kTileRows) * kTileRows;
    }
    seg_s[S] = start;
    for (int s = 0; s <= S; ++s) ws.seg[s] = (int)seg_s[s];
    ws.seg[kMaxS + 1] = raw_at_species[S];  // real atoms
  }
  __syncthreads();
  // bin_start = raw prefix + the padding of the preceding species segments
  if (in_smem) {
    for (int b = t; b < nb; b += 1024) {  // coalesced
      int sp = 0;
#pragma unroll
      for (int q = 1; q < kMaxS; ++q) sp += (q < S && b >= q * TC) ? 1 : 0;
      ws.bin_start[b] = s_bins[b] + (int)(seg_s[sp] - raw_at_species[sp]);
    }
  } else {
    int run = run0;
    int sp = TC > 0 ? b0 / TC : 0, sp_start = sp * TC;
    int shift = (sp < S) ? (int)(seg_s[sp] - raw_at_species[sp]) : 0;
    for (int b = b0; b < b1; ++b) {
      if (b == sp_start + TC) {
        ++sp;
        sp_start += TC;
        shift = (int)(seg_s[sp] - raw_at_species[sp]);
      }
      const int c = ws.bin_count[b];
      ws.bin_start[b] = run + shift;
      ws.bin_len[b] = c;
      run += c;
    }
  }
  if (t == 0) ws.bin_start[nb] = (int)seg_s[S];
  // padding rows at the end of each species segment
  for (int s = 0; s < S; ++s) {
    const int first_pad = (int)seg_s[s] + (raw_at_species[s + 1] - raw_at_species[s]);
    for (int r = first_pad + t; r < seg_s[s + 1]; r += 1024) {
      ws.row_atom[r] = -1;
      ws.pos4[r] = make_float4(0.f, 0.f, 0.f, __int_as_float(s));
      ws.row_info[r] = 0;
      ws.row_cell[r] = 0;
      for (int sp = 0; sp < S; ++sp) {
        ws.cnt_r[(size_t)r * kMaxS + sp] = 0;
        ws.cnt_a[(size_t)r * kMaxS + sp] = 0;
      }
    }
  }
}

__global__ void __launch_bounds__(1024) k_scan(const EvalIO* __restrict__ io, int S, Workspace ws) {
  extern __shared__ int s_bins[];  // [kScanSmemBins]: counts, then raw starts
  scan_bins(io, S, ws, s_bins, kScanSmemBins);
}

__device__ __forceinline__ void scatter_atoms(const EvalIO* __restrict__ io, const Workspace& ws, long long tid0,
                                              long long stride) {
  const long long n = io->n_atoms;
  for (long long a = tid0; a < n; a += stride) {
    const int row = ws.bin_start[ws.atom_bin[a]] + ws.atom_slot[a];
    if (NNP_IN(row, ws.max_rows, ws.flags)) ws.row_atom[row] = (int)a;
  }
}

__global__ void k_scatter(const EvalIO* __restrict__ io, Workspace ws) {
  scatter_atoms(io, ws, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// Warp per bin: order the bin's atoms by input index (ranks by comparison),
// then write the row arrays.  Bins with more than kSortCap atoms keep slot
// order (flagged; results stay correct, only summation order differs).
constexpr int kSortCap = 256;
// warp0: this warp's first bin, wstride: warps over all bins, sw: the warp's
// kSortCap ints of shared memory
__device__ __forceinline__ void sort_bins(const EvalIO* __restrict__ io, int S, int sort, const Workspace& ws,
                                          int warp0, int wstride, int* sw) {
  const int lane = threadIdx.x & 31;
  const int nb = S * io->total_cells;
  for (int b = warp0; b < nb; b += wstride) {
    const int start = ws.bin_start[b];
    const int cnt = ws.bin_len[b];
    if (lane == 0) ws.bin_count[b] = 0;  // ready for the next evaluation
    if (cnt == 0) continue;
    const bool do_sort = sort && cnt <= kSortCap;
    if (sort && !do_sort && lane == 0) atomicOr(&ws.flags[kFlagBinOverflow], 1);
    if (do_sort) {
      for (int k = lane; k < cnt; k += 32) sw[k] = ws.row_atom[start + k];
      __syncwarp();
      // each lane writes the rows of the atoms it ranked (no re-read of row_atom)
      for (int k = lane; k < cnt; k += 32) {
        const int a = sw[k];
        int rank = 0;
        for (int q = 0; q < cnt; ++q) rank += sw[q] < a;
        const int row = start + rank;
        ws.row_atom[row] = a;
        ws.pos4[row] = ws.atom_off[a];
        ws.row_info[row] = ws.atom_sys[a];
        ws.row_cell[row] = ws.atom_cell[a];
      }
    } else {
      for (int k = lane; k < cnt; k += 32) {
        const int row = start + k;
        const int a = ws.row_atom[row];
        ws.pos4[row] = ws.atom_off[a];
        ws.row_info[row] = ws.atom_sys[a];
        ws.row_cell[row] = ws.atom_cell[a];
      }
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(256) k_binsort(const EvalIO* __restrict__ io, int S, int sort,
                                                 Workspace ws) {
  __shared__ int sm[8][kSortCap];
  const int w = threadIdx.x >> 5;
  sort_bins(io, S, sort, ws, (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5),
            (int)((gridDim.x * blockDim.x) >> 5), sm[w]);
}

// Small systems: the four steps in one block of 1024 threads, block barriers
// between them (global writes of the block are visible after a barrier).
__global__ void __launch_bounds__(1024) k_cells_small(const EvalIO* __restrict__ io,
                                                      const SysDesc* __restrict__ sys,
                                                      const signed char* __restrict__ zlut, int S, int sort,
                                                      Workspace ws) {
  extern __shared__ int s_dyn_cells[];  // [kScanSmemBinsSmall] scan, then [32][kSortCap] sort
  bin_atoms(io, sys, zlut, ws, threadIdx.x, 1024, nullptr);
  __syncthreads();
  scan_bins(io, S, ws, s_dyn_cells, kScanSmemBinsSmall);
  __syncthreads();
  scatter_atoms(io, ws, threadIdx.x, 1024);
  __syncthreads();
  sort_bins(io, S, sort, ws, threadIdx.x >> 5, 32, s_dyn_cells + (threadIdx.x >> 5) * kSortCap);
}

// Warp per cell (grid-stride over the cells of every system).  For each
// neighbour species, the atoms of the 27 virtual cells around the cell
// (periodic images by the virtual cell offset m in {-1,0,1}^3, shift
// sum_d m_d cv_d) are staged in the warp's shared window as positions relative
// to the cell's corner plus their list entry.  A candidate (j, m) is kept if
// |off_j + shift(m) - off_i| < rc_r and it is not the atom itself; within a
// species, entries inside rc_a come first in the row's segment, then the
// radial-only ones (their order is free).  Counts are clamped to what the
// list holds, so readers never run past it; the unclamped maxima raise the
// overflow flags (one update per CTA).  Padding rows get zero counts from
// k_scan.
//
// Two ways through a cell.  The group path (windows that fit kNbrWin): rows
// in groups of up to 16 with 2-32 lanes per row, each lane testing a share of
// the window's 32-candidate chunks; hit counts are scanned over a row's lanes
// so every entry goes straight to its place.  The lane-per-row path (larger
// windows): one lane per row over windows of kNbrWin, radial-only entries
// parked at the end of the list and moved down once the species is done.
// Both keep the hit masks of a lane in shared-memory slots and write the hits
// with one loop whose step count is the same for the whole warp.  SB >= S
// bounds the per-species register arrays and scans (2, 4 or 8).  WIN is the
// window (512; 1024 for small systems, with row groups of at most 8, and 2048
// for a system of one cell, with groups of at most 4, so that a lane still
// tests at most 8 chunks).  split > 1 spreads a cell's row groups over that
// many warps, for systems with fewer cells than the GPU has warps.
template <int SB, int WIN>
__global__ void __launch_bounds__(kNbrThreads, 5) k_neighbors(const EvalIO* __restrict__ io,
                                                          const SysDesc* __restrict__ sys,
                                                          DescParams P, Workspace ws, int split, int dyn) {
  constexpr int NCH = WIN / 32;                                       // window chunks
  constexpr int WF = 3 * NCH * kNbrChunkStride + WIN + 16 * 32;       // shared floats per warp
  constexpr int GR = WIN > 1024 ? 4 : (WIN > 512 ? 8 : 16);           // rows per group
  constexpr unsigned F = 0xffffffffu;
  __shared__ int s_mx[3];  // maxima of the CTA's row counts; warps done
  extern __shared__ float4 s_dyn[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // per warp: the candidate window as arrays of x, y, z (chunks of 32 at a
  // stride of 36 floats, so that the lanes of a row, reading different
  // chunks, hit different banks) and of list entries, then the 16 hit-mask
  // slots of the group path
  float* wx = reinterpret_cast<float*>(s_dyn) + (size_t)wib * WF;
  float* wy = wx + NCH * kNbrChunkStride;
  float* wz = wy + NCH * kNbrChunkStride;
  int* we = reinterpret_cast<int*>(wz + NCH * kNbrChunkStride);
  unsigned* hmask = reinterpret_cast<unsigned*>(we + WIN);
  const int TC = io->total_cells, nsys = io->n_sys, S = P.S, cap = ws.cap_r;
  const float rcr2 = P.rc_r * P.rc_r, rca2 = P.rc_a * P.rc_a;
  const f2 nrc2 = f2_make(-rcr2, -rcr2), nra2 = f2_make(-rca2, -rca2);
  int mx_r = 0, mx_a = 0;  // largest unclamped row counts seen by this lane
  const int wpb = blockDim.x >> 5;
  (void)wib;
  if (threadIdx.x < 3) s_mx[threadIdx.x] = 0;
  __syncthreads();
  // cells (each split into `split` parts) from the work queue
  WorkQueue wq(ws.queue + kQNbr, dyn != 0);
  for (int vg = wq.first(); vg < TC * split; vg = wq.next(lane)) {
    const int g = vg / split, part = vg - g * split;
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sys[mid].cell_base <= g) lo = mid; else hi = mid - 1;
    }
    const SysDesc& sd = sys[lo];
    const int nc0 = sd.nc[0], nc1 = sd.nc[1], nc2 = sd.nc[2];
    const int lc = g - sd.cell_base;
    const int cz = lc % nc2, cy = (lc / nc2) % nc1, cx = lc / (nc1 * nc2);
    // rows of this cell: lane s < S holds species s's bin (first row, length)
    int rst = 0, rln = 0;
    if (lane < S) {
      const int b = lane * TC + g;
      rst = ws.bin_start[b];
      rln = ws.bin_len[b];
    }
    int rpre = rln;  // inclusive prefix over species
#pragma unroll
    for (int o = 1; o < SB; o <<= 1) {
      const int y = __shfl_up_sync(F, rpre, o);
      if (lane >= o) rpre += y;
    }
    const int nrows = __shfl_sync(F, rpre, SB - 1);
    if (nrows == 0) continue;
    // virtual cell v = lane (< 27): local index of the real cell, or -1 outside an open boundary
    int vcell = -1;
    if (lane < 27) {
      int v[3] = {cx + lane / 9 - 1, cy + (lane / 3) % 3 - 1, cz + lane % 3 - 1};
      const int ncv[3] = {nc0, nc1, nc2};
      bool ok = true;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (v[c] < 0 || v[c] >= ncv[c]) {
          if (sd.periodic) v[c] = (v[c] + ncv[c]) % ncv[c];
          else ok = false;
        }
      }
      if (ok) vcell = (v[0] * nc1 + v[1]) * nc2 + v[2];
    }
    // bins of the 27 virtual cells for every species (lane v), their exclusive
    // offsets within the species' flattened neighbourhood, and its size
    int bst[SB], bln[SB], bex[SB], tot[SB];
    int max_tot = 0, sum_tot = 0;  // sum of the windows, each rounded up to whole chunks
#pragma unroll
    for (int sp = 0; sp < SB; ++sp) {
      bst[sp] = 0;
      bln[sp] = 0;
      if (sp < S && vcell >= 0) {
        const int b = sp * TC + sd.cell_base + vcell;
        bst[sp] = ws.bin_start[b];
        bln[sp] = ws.bin_len[b];
      }
      int incl = bln[sp];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(F, incl, o);
        if (lane >= o) incl += y;
      }
      tot[sp] = __shfl_sync(F, incl, 31);
      bex[sp] = incl - bln[sp];
      max_tot = max(max_tot, tot[sp]);
      sum_tot += (tot[sp] + 31) & ~31;
    }
    // per-species register arrays are read with constant indices only
    auto pick = [&](const int (&a)[SB], int sp) {
      int x = a[0];
#pragma unroll
      for (int t = 1; t < SB; ++t)
        if (sp == t) x = a[t];
      return x;
    };
    // stage the window [w0, w0 + wn) of species sp's neighbourhood: lane v <
    // 27 copies the atoms of virtual cell v (shifted by its image offset) to
    // their places bex[v] + k; the loads of the 27 cells are independent
    const float3 vs = cell_shift(lane / 9 - 1, (lane / 3) % 3 - 1, lane % 3 - 1, sd);
    const float vsx = vs.x, vsy = vs.y, vsz = vs.z;
    auto stage = [&](int sp, int w0, int wn, int db) {
      const int bex_s = pick(bex, sp), bst_s = pick(bst, sp), bln_s = pick(bln, sp);
      const int k0 = max(0, w0 - bex_s), k1 = min(bln_s, w0 + wn - bex_s);
      __syncwarp();  // the previous window has been read
#pragma unroll 4
      for (int k = k0; k < k1; ++k) {
        if (!(NNP_IN(bst_s + k, ws.max_rows, ws.flags) && NNP_IN(db + bex_s + k - w0, WIN, ws.flags))) break;
        const float4 pj = ws.pos4[bst_s + k];
        const int gi = db + bex_s + k - w0, ci = (gi >> 5) * kNbrChunkStride + (gi & 31);
        wx[ci] = pj.x + vsx;
        wy[ci] = pj.y + vsy;
        wz[ci] = pj.z + vsz;
        we[gi] = pack_nbr(bst_s + k, lane);
      }
      __syncwarp();
    };
    // row of lane position q (species-major within the cell)
    auto row_of = [&](int q) {
      int row = 0;
#pragma unroll
      for (int s = 0; s < SB; ++s) {
        const int inc = __shfl_sync(F, rpre, s), len = __shfl_sync(F, rln, s), st = __shfl_sync(F, rst, s);
        if (q >= inc - len && q < inc) row = st + (q - (inc - len));
      }
      return row;
    };
    // hit masks of the 32 candidates of the chunk starting at k0 (a multiple
    // of 32; the window ends at wn) against the row at -(nx, ny, nz).  Bit k
    // is the sign of r^2 - rc^2 (exact: both are near-equal normal floats
    // or clearly ordered), shifted in by one funnel shift per candidate.
    auto masks = [&](const f2 nx, const f2 ny, const f2 nz, int k0, int wn, unsigned& hr, unsigned& ha) {
      const int cb = (k0 >> 5) * kNbrChunkStride;
      unsigned r = 0u, a = 0u;
#pragma unroll
      for (int j = 0; j < 8; ++j) {  // past wn: stale window data, masked below
        const float4 X = *reinterpret_cast<const float4*>(wx + cb + 4 * j);
        const float4 Y = *reinterpret_cast<const float4*>(wy + cb + 4 * j);
        const float4 Z = *reinterpret_cast<const float4*>(wz + cb + 4 * j);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const f2 dx = f2_add(u ? f2_make(X.z, X.w) : f2_make(X.x, X.y), nx);
          const f2 dy = f2_add(u ? f2_make(Y.z, Y.w) : f2_make(Y.x, Y.y), ny);
          const f2 dz = f2_add(u ? f2_make(Z.z, Z.w) : f2_make(Z.x, Z.y), nz);
          const f2 r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
          const float2 dr = f2_split(f2_add(r2, nrc2)), da = f2_split(f2_add(r2, nra2));
          r = __funnelshift_l(__float_as_uint(dr.x), r, 1);
          r = __funnelshift_l(__float_as_uint(dr.y), r, 1);
          a = __funnelshift_l(__float_as_uint(da.x), a, 1);
          a = __funnelshift_l(__float_as_uint(da.y), a, 1);
        }
      }
      hr = __brev(r);  // candidate k at bit k
      ha = __brev(a);
      if (wn - k0 < 32) hr &= (1u << (wn - k0)) - 1u;
      ha &= hr;
    };

    if (max_tot <= WIN) {
      // ---- group path: rows in groups of up to 16, h = 32 / 2^ceil(log2(rows))
      // lanes per row (h >= 2), lane p of a row testing its share of the
      // window's 32-candidate chunks.  Hit counts are scanned over the h
      // lanes of the row, so every entry goes straight to its final place
      // (angular ones first, both kinds in window order).  When the windows
      // of all species fit, they are staged once for all groups.
      if (GR * part >= nrows) continue;  // split > 1: this part has no row group
      const bool all_fit = sum_tot <= WIN;
      if (all_fit) {
        int wb = 0;
        for (int sp = 0; sp < S; ++sp) {
          const int wn = pick(tot, sp);
          stage(sp, 0, wn, wb);
          wb += (wn + 31) & ~31;
        }
      }
      for (int r0 = GR * part; r0 < nrows; r0 += GR * split) {
        const int rg = min(GR, nrows - r0);
        const int lh = rg > 8 ? 1 : (rg > 4 ? 2 : (rg > 2 ? 3 : (rg > 1 ? 4 : 5)));  // log2 h
        const int h = 1 << lh;
        const int ql = lane >> lh, p = lane & (h - 1);
        const bool has = ql < rg;
        const int row = row_of(r0 + ql);
        const float4 pi = has ? ws.pos4[row] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int row_sp = pos4_species(pi);
        const f2 nx = f2_make(-pi.x, -pi.x), ny = f2_make(-pi.y, -pi.y), nz = f2_make(-pi.z, -pi.z);
        int* lr = ws.nbr_r + (size_t)row * cap;
        int nr = 0, tot_r = 0, tot_a = 0, wb = 0;
        for (int sp = 0; sp < S; ++sp) {
          const int wn = pick(tot, sp);
          if (wn == 0) {  // no atom of this species near the cell (warp-uniform)
            if (has && p == 0) {
              ws.cnt_r[(size_t)row * kMaxS + sp] = 0;
              ws.cnt_a[(size_t)row * kMaxS + sp] = 0;
            }
            continue;
          }
          if (!all_fit) stage(sp, 0, wn, 0);
          const int nch = (wn + 31) >> 5;
          const int ch0 = (p * nch) >> lh, ch1 = ((p + 1) * nch) >> lh;
          // the row itself: image 0 in virtual cell 13 of its own species
          const int ex13 = __shfl_sync(F, pick(bex, sp), 13), st13 = __shfl_sync(F, pick(bst, sp), 13);
          const int self_k = (row_sp == sp) ? ex13 + (row - st13) : -1;
          // hit masks of the lane's chunks go to the warp's mask buffer, slot
          // 2i for the angular hits of chunk ch0 + i and 2i + 1 for the
          // radial-only ones, so one flat loop per lane then walks all of its
          // hits (the warp pays the largest hit count of a lane, not the sum
          // over chunks of the per-chunk largest)
          int na_me = 0, nro_me = 0;
          unsigned nzs = 0u;  // slots with hits
#pragma unroll 1
          for (int i = 0; i < (has ? ch1 - ch0 : 0); ++i) {
            const int ch = ch0 + i;
            unsigned hr, ha;
            masks(nx, ny, nz, wb + ch * 32, wb + wn, hr, ha);
            if ((self_k >> 5) == ch) {
              hr &= ~(1u << (self_k & 31));
              ha &= hr;
            }
            hmask[(2 * i) * 32 + lane] = ha;
            hmask[(2 * i + 1) * 32 + lane] = hr & ~ha;
            nzs |= (ha ? 1u : 0u) << (2 * i);
            nzs |= ((hr & ~ha) ? 1u : 0u) << (2 * i + 1);
            na_me += __popc(ha);
            nro_me += __popc(hr & ~ha);
          }
          // offsets of the lane's hits within the row's segment
          int ia = na_me, ir = nro_me;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            if (o >= h) break;
            const int ya = __shfl_up_sync(F, ia, o, h), yr = __shfl_up_sync(F, ir, o, h);
            if (p >= o) {
              ia += ya;
              ir += yr;
            }
          }
          const int NA = __shfl_sync(F, ia, h - 1, h), NRO = __shfl_sync(F, ir, h - 1, h);
          int apos = nr + ia - na_me, rpos = nr + NA + ir - nro_me;
          {
            // one step per hit, the same step count for the whole warp (a
            // nested data-dependent loop would let the lanes drift apart and
            // run one after another); nz marks the lane's slots still holding hits
            const int steps = __reduce_max_sync(F, (unsigned)(na_me + nro_me));
            unsigned nz = has ? nzs : 0u, cur = 0u;
            int base = 0;
            bool ang = true;
            for (int it = 0; it < steps; ++it) {
              if (cur == 0u && nz != 0u) {
                const int m = __ffs(nz) - 1;
                nz &= nz - 1u;
                cur = hmask[m * 32 + lane];
                base = wb + (ch0 + (m >> 1)) * 32;
                ang = (m & 1) == 0;
              }
              if (cur != 0u) {
                const int k = __ffs(cur) - 1;
                cur &= cur - 1u;
                const int e = we[base + k];
                const int q = ang ? apos : rpos;
                if (q < cap) lr[q] = e;
                apos += ang ? 1 : 0;
                rpos += ang ? 0 : 1;
              }
            }
          }
          __syncwarp();  // the mask buffer and the window are rewritten next
          // counts clamped to what the list holds, so readers never run past it
          const int keep = max(0, min(NA + NRO, cap - nr));
          if (has && p == 0) {
            ws.cnt_r[(size_t)row * kMaxS + sp] = keep;
            ws.cnt_a[(size_t)row * kMaxS + sp] = min(NA, keep);
          }
          nr += keep;
          tot_r += NA + NRO;
          tot_a += NA;
          if (all_fit) wb += (wn + 31) & ~31;
        }
        if (has && p == 0) {
          mx_r = max(mx_r, tot_r);
          mx_a = max(mx_a, tot_a);
        }
      }
      continue;
    }

    // ---- lane per row (cells of many rows, or windows beyond kNbrWin): the
    // species' neighbourhood in windows of kNbrWin candidates, each tested in
    // halves of 8 chunks whose hit masks go to the mask slots, then written
    // by one flat loop with a warp-uniform step count.  Angular entries go to
    // the front of the row's segment, radial-only ones are parked at the end
    // of the list and moved behind them once the species is done.
    for (int r0 = 32 * part; r0 < nrows; r0 += 32 * split) {
      const int q = r0 + lane;
      const bool has = q < nrows;
      const int row = row_of(q);
      const float4 pi = has ? ws.pos4[row] : make_float4(0.f, 0.f, 0.f, 0.f);
      const int row_sp = pos4_species(pi);
      const f2 nx = f2_make(-pi.x, -pi.x), ny = f2_make(-pi.y, -pi.y), nz = f2_make(-pi.z, -pi.z);
      int* lr = ws.nbr_r + (size_t)row * cap;
      int nr = 0, tot_r = 0, tot_a = 0;  // written entries; all entries found
      for (int sp = 0; sp < S; ++sp) {
        const int total = pick(tot, sp);
        const int ex13 = __shfl_sync(F, pick(bex, sp), 13), st13 = __shfl_sync(F, pick(bst, sp), 13);
        const int self_k = (has && row_sp == sp) ? ex13 + (row - st13) : -1;
        int wa = 0, wro = 0, ka = 0, kro = 0;  // written / found: angular, radial-only
        for (int w0 = 0; w0 < total; w0 += WIN) {
          const int wn = min(WIN, total - w0);
          stage(sp, w0, wn, 0);
          for (int h0 = 0; h0 < wn; h0 += 256) {
            const int nch = (min(256, wn - h0) + 31) >> 5;
            int n_me = 0;
            unsigned nzs = 0u;
#pragma unroll 1
            for (int i = 0; i < (has ? nch : 0); ++i) {
              const int k0 = h0 + 32 * i;
              unsigned hr, ha;
              masks(nx, ny, nz, k0, wn, hr, ha);
              const int sk = self_k - w0 - k0;  // the row itself, image 0
              if (self_k >= 0 && sk >= 0 && sk < 32) {
                hr &= ~(1u << sk);
                ha &= hr;
              }
              hmask[(2 * i) * 32 + lane] = ha;
              hmask[(2 * i + 1) * 32 + lane] = hr & ~ha;
              nzs |= (ha ? 1u : 0u) << (2 * i);
              nzs |= ((hr & ~ha) ? 1u : 0u) << (2 * i + 1);
              n_me += __popc(hr);
            }
            const int steps = __reduce_max_sync(F, (unsigned)n_me);
            unsigned nzl = has ? nzs : 0u, cur = 0u;
            int base = 0;
            bool ang = true;
            for (int it = 0; it < steps; ++it) {
              if (cur == 0u && nzl != 0u) {
                const int m = __ffs(nzl) - 1;
                nzl &= nzl - 1u;
                cur = hmask[m * 32 + lane];
                base = h0 + (m >> 1) * 32;
                ang = (m & 1) == 0;
              }
              if (cur != 0u) {
                const int k = __ffs(cur) - 1;
                cur &= cur - 1u;
                const int e = we[base + k];
                const bool room = nr + wa + wro < cap;
                if (ang) {
                  if (room) lr[nr + wa++] = e;
                  ++ka;
                } else {
                  if (room) lr[cap - 1 - wro++] = e;
                  ++kro;
                }
              }
            }
            __syncwarp();  // the mask slots are rewritten by the next half
          }
        }
        if (has) {
          // bring the parked radial-only entries down behind the angular ones
          const int m = min(wro, cap - wro - (nr + wa));
          for (int k = 0; k < m; ++k) lr[nr + wa + k] = lr[cap - 1 - k];
          ws.cnt_r[(size_t)row * kMaxS + sp] = wa + wro;
          ws.cnt_a[(size_t)row * kMaxS + sp] = wa;
        }
        nr += wa + wro;
        tot_r += ka + kro;
        tot_a += ka;
      }
      if (has) {
        mx_r = max(mx_r, tot_r);
        mx_a = max(mx_a, tot_a);
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    mx_r = max(mx_r, __shfl_xor_sync(F, mx_r, o));
    mx_a = max(mx_a, __shfl_xor_sync(F, mx_a, o));
  }
  queue_warp_done(wq, lane);
  // the CTA's last warp to finish publishes the maxima (no block barrier, so
  // warps that finish early do not wait)
  if (lane == 0) {
    atomicMax(&s_mx[0], mx_r);
    atomicMax(&s_mx[1], mx_a);
    __threadfence_block();
    if (atomicAdd(&s_mx[2], 1) == wpb - 1) {
      const int r = atomicMax(&s_mx[0], 0), a = atomicMax(&s_mx[1], 0);
      if (r | a) {
        atomicMax(&ws.flags[kFlagMaxNbrR], r);
        atomicMax(&ws.flags[kFlagMaxNbrA], a);
        if (r > ws.cap_r) atomicOr(&ws.flags[kFlagOverflowR], 1);
        if (a > ws.cap_a) atomicOr(&ws.flags[kFlagOverflowA], 1);
      }
    }
  }
}

size_t neighbors_smem(int win) {
  return sizeof(float) * (size_t)(3 * (win / 32) * kNbrChunkStride + win + 16 * 32) * (kNbrThreads / 32);
}

cudaError_t neighbors_set_smem_limits() {
  cudaError_t e = cudaFuncSetAttribute(k_scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(int) * kScanSmemBins));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cells_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(int) * kScanSmemBinsSmall));
  const int s1 = (int)neighbors_smem(kNbrWin), s2 = (int)neighbors_smem(kNbrWinSmall);
  const int s3 = (int)neighbors_smem(kNbrWinTiny);
#define NSM(sb)                                                                                                   \
  if (e == cudaSuccess)                                                                                           \
    e = cudaFuncSetAttribute(k_neighbors<sb, kNbrWin>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);          \
  if (e == cudaSuccess)                                                                                           \
    e = cudaFuncSetAttribute(k_neighbors<sb, kNbrWinSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2);     \
  if (e == cudaSuccess)                                                                                           \
    e = cudaFuncSetAttribute(k_neighbors<sb, kNbrWinTiny>, cudaFuncAttributeMaxDynamicSharedMemorySize, s3);
  NSM(2) NSM(4) NSM(8)
#undef NSM
  return e;
}

void launch_neighbors(int grid, cudaStream_t st, const EvalIO* io, const SysDesc* sys, const DescParams& P,
                      const Workspace& ws, long long rows, long long cells, int nsm, int mode) {
  const int dyn = mode & 1;
  if (rows > kNbrRowsSmall) {  // warp per cell (mode & 2: per half cell), 512-candidate windows
    const size_t sm = neighbors_smem(kNbrWin);
    const int sp = (mode & 2) ? 2 : 1;
    if (P.S <= 2) k_neighbors<2, kNbrWin><<<grid, kNbrThreads, sm, st>>>(io, sys, P, ws, sp, dyn);
    else if (P.S <= 4) k_neighbors<4, kNbrWin><<<grid, kNbrThreads, sm, st>>>(io, sys, P, ws, sp, dyn);
    else k_neighbors<8, kNbrWin><<<grid, kNbrThreads, sm, st>>>(io, sys, P, ws, sp, dyn);
    return;
  }
  if (cells == 1) {  // one cell: its 27 images in 2048-candidate windows, row groups of 4 over up to 32 warps
    const int split = (int)std::max(1LL, std::min(32LL, (rows + 3) / 4));
    const size_t sm = neighbors_smem(kNbrWinTiny);
    if (P.S <= 2) k_neighbors<2, kNbrWinTiny><<<(split + 3) / 4, kNbrThreads, sm, st>>>(io, sys, P, ws, split, dyn);
    else if (P.S <= 4) k_neighbors<4, kNbrWinTiny><<<(split + 3) / 4, kNbrThreads, sm, st>>>(io, sys, P, ws, split, dyn);
    else k_neighbors<8, kNbrWinTiny><<<(split + 3) / 4, kNbrThreads, sm, st>>>(io, sys, P, ws, split, dyn);
    return;
  }
  // small systems: 1024-candidate windows, each cell's row groups over up to 8 warps
  const long long target = 8LL * nsm;  // warps to aim for
  const int split = (int)std::max(1LL, std::min(8LL, (target + cells - 1) / std::max(1LL, cells)));
  const long long warps = cells * split;
  const int g = (int)std::max(1LL, (warps + kNbrThreads / 32 - 1) / (kNbrThreads / 32));
  const size_t sm = neighbors_smem(kNbrWinSmall);
  if (P.S <= 2) k_neighbors<2, kNbrWinSmall><<<g, kNbrThreads, sm, st>>>(io, sys, P, ws, split, dyn);
  else if (P.S <= 4) k_neighbors<4, kNbrWinSmall><<<g, kNbrThreads, sm, st>>>(io, sys, P, ws, split, dyn);
  else k_neighbors<8, kNbrWinSmall><<<g, kNbrThreads, sm, st>>>(io, sys, P, ws, split, dyn);
}

}  // namespace nnp
