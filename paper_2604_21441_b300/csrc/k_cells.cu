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
//   k_neighbors  warp per row: 27 neighbour cells x S species, lists grouped
//                by neighbour species
#include "nnp_internal.cuh"

namespace nnp {

__global__ void k_bin(const EvalIO* __restrict__ io, const SysDesc* __restrict__ sys,
                      const signed char* __restrict__ zlut, Workspace ws) {
  const long long n = io->n_atoms;
  const int TC = io->total_cells;
  const int nsys = io->n_sys;
  const long long tid0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (tid0 < nsys) io->energies[tid0] = 0.0;
  for (long long a = tid0; a < n; a += stride) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (sys[mid].atom_begin <= a) lo = mid; else hi = mid - 1;
    }
    const SysDesc& sd = sys[lo];
    double p[3] = {io->pos[3 * a], io->pos[3 * a + 1], io->pos[3 * a + 2]};
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
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double x = p[c] - sd.origin[c];
      if (sd.periodic) {
        x -= sd.L[c] * floor(x / sd.L[c]);
        if (x >= sd.L[c]) x -= sd.L[c];
        if (x < 0.0) x = 0.0;
      }
      int kk = (int)floor(x / sd.ell[c]);
      kk = kk < 0 ? 0 : (kk >= sd.nc[c] ? sd.nc[c] - 1 : kk);
      k[c] = kk;
      off[c] = (float)(x - kk * sd.ell[c]);
    }
    const int cell = (k[0] * sd.nc[1] + k[1]) * sd.nc[2] + k[2];
    const int bin = s * TC + sd.cell_base + cell;
    ws.atom_slot[a] = atomicAdd(&ws.bin_count[bin], 1);
    ws.atom_bin[a] = bin;
    ws.atom_off[a] = make_float4(off[0], off[1], off[2],
                                 __int_as_float((int)(((unsigned)a << 3) | (unsigned)s)));
    ws.atom_cell[a] = k[0] | (k[1] << 10) | (k[2] << 20);
    ws.atom_sys[a] = lo;
    io->forces[3 * a] = 0.0;
    io->forces[3 * a + 1] = 0.0;
    io->forces[3 * a + 2] = 0.0;
  }
}

// Single CTA of 1024 threads.  bin_start[b] = first row of bin b, with each
// species segment starting on a multiple of kTileRows; bin_len keeps counts.
__global__ void __launch_bounds__(1024) k_scan(const EvalIO* __restrict__ io, int S, Workspace ws) {
  __shared__ int warp_tot[32];
  __shared__ long long seg_s[kMaxS + 2];
  __shared__ int raw_at_species[kMaxS + 1];
  const int nb = S * io->total_cells;
  const int TC = io->total_cells;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int chunk = (nb + 1023) / 1024;
  const int b0 = t * chunk, b1 = min(nb, b0 + chunk);
  int sum = 0;
  for (int b = b0; b < b1; ++b) sum += ws.bin_count[b];
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
  int run = warp_tot[wid] + incl - sum;
  for (int b = b0; b < b1; ++b) {
    int c = ws.bin_count[b];
    ws.bin_start[b] = run;   // raw prefix (no padding yet)
    ws.bin_len[b] = c;
    run += c;
    if (b % TC == 0) raw_at_species[b / TC] = ws.bin_start[b];
  }
  if (b1 == nb && b0 < b1) raw_at_species[S] = run;
  if (nb == 0 && t == 0) raw_at_species[S] = 0;
  __syncthreads();
  if (t == 0) {
    long long start = 0;
    for (int s = 0; s < S; ++s) {
      seg_s[s] = start;
      const int cnt = raw_at_species[s + 1] - raw_at_species[s];
      start = ((start + cnt + kTileRows - 1) / kTileRows) * kTileRows;
    }
    seg_s[S] = start;
    for (int s = 0; s <= S; ++s) ws.seg[s] = (int)seg_s[s];
    ws.seg[kMaxS + 1] = raw_at_species[S];  // real atoms
  }
  __syncthreads();
  for (int b = t; b < nb; b += 1024) {
    const int s = b / TC;
    ws.bin_start[b] += (int)(seg_s[s] - raw_at_species[s]);
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
    }
  }
}

__global__ void k_scatter(const EvalIO* __restrict__ io, Workspace ws) {
  const long long n = io->n_atoms;
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < n;
       a += (long long)gridDim.x * blockDim.x) {
    const int row = ws.bin_start[ws.atom_bin[a]] + ws.atom_slot[a];
    ws.row_atom[row] = (int)a;
  }
}

// Warp per bin: order the bin's atoms by input index (ranks by comparison),
// then write the row arrays.  Bins with more than kSortCap atoms keep slot
// order (flagged; results stay correct, only summation order differs).
constexpr int kSortCap = 256;
__global__ void __launch_bounds__(256) k_binsort(const EvalIO* __restrict__ io, int S, int sort,
                                                 Workspace ws) {
  __shared__ int sm[8][kSortCap];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nb = S * io->total_cells;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb;
       b += (gridDim.x * blockDim.x) >> 5) {
    const int start = ws.bin_start[b];
    const int cnt = ws.bin_len[b];
    if (lane == 0) ws.bin_count[b] = 0;  // ready for the next evaluation
    if (cnt == 0) continue;
    const bool do_sort = sort && cnt <= kSortCap;
    if (sort && !do_sort && lane == 0) atomicOr(&ws.flags[kFlagBinOverflow], 1);
    if (do_sort) {
      for (int k = lane; k < cnt; k += 32) sm[w][k] = ws.row_atom[start + k];
      __syncwarp();
      for (int k = lane; k < cnt; k += 32) {
        const int a = sm[w][k];
        int rank = 0;
        for (int q = 0; q < cnt; ++q) rank += sm[w][q] < a;
        const int row = start + rank;
        ws.row_atom[row] = a;
      }
      __syncwarp();
    }
    for (int k = lane; k < cnt; k += 32) {
      const int row = start + k;
      const int a = ws.row_atom[row];
      ws.pos4[row] = ws.atom_off[a];
      ws.row_info[row] = ws.atom_sys[a];
      ws.row_cell[row] = ws.atom_cell[a];
    }
    __syncwarp();
  }
}

// Warp per row.  Candidates: for each neighbour species s', the atoms of the
// 27 virtual cells around the row's cell, flattened into one index space so
// that all 32 lanes test candidates.  A candidate (j, image m) is kept if
// |off_j - off_i + m*ell| < rc_r and it is not the atom itself.  Entries
// within rc_a go straight to the row's list; radial-only entries wait in a
// per-warp shared buffer and are appended after the species' angular ones.
__global__ void __launch_bounds__(256) k_neighbors(const EvalIO* __restrict__ io,
                                                   const SysDesc* __restrict__ sys,
                                                   DescParams P, Workspace ws) {
  __shared__ int s_start[8][32];
  __shared__ int s_excl[8][33];
  extern __shared__ int s_stage[];  // [8][cap_r]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int* stage = s_stage + (size_t)w * ws.cap_r;
  const int rows = ws.seg[P.S];
  const int TC = io->total_cells;
  const float rcr2 = P.rc_r * P.rc_r, rca2 = P.rc_a * P.rc_a;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows;
       row += (gridDim.x * blockDim.x) >> 5) {
    int* cr = ws.cnt_r + (size_t)row * kMaxS;
    int* ca = ws.cnt_a + (size_t)row * kMaxS;
    if (ws.row_atom[row] < 0) {
      if (lane < kMaxS) { cr[lane] = 0; ca[lane] = 0; }
      continue;
    }
    const float4 pi = ws.pos4[row];
    const SysDesc& sd = sys[ws.row_info[row]];
    const int pc = ws.row_cell[row];
    const int cx = pc & 1023, cy = (pc >> 10) & 1023, cz = (pc >> 20) & 1023;
    const float ell[3] = {sd.ellf[0], sd.ellf[1], sd.ellf[2]};
    int* lr = ws.nbr_r + (size_t)row * ws.cap_r;
    int nr = 0, na = 0;  // entries found so far (all species), may exceed capacity
    for (int sp = 0; sp < P.S; ++sp) {
      int len = 0, st = 0;
      if (lane < 27) {
        int v[3] = {cx + lane / 9 - 1, cy + (lane / 3) % 3 - 1, cz + lane % 3 - 1};
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (v[c] < 0 || v[c] >= sd.nc[c]) {
            if (sd.periodic) v[c] = (v[c] + sd.nc[c]) % sd.nc[c];
            else ok = false;
          }
        }
        if (ok) {
          const int bin = sp * TC + sd.cell_base + (v[0] * sd.nc[1] + v[1]) * sd.nc[2] + v[2];
          st = ws.bin_start[bin];
          len = ws.bin_len[bin];
        }
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      s_start[w][lane] = st;
      s_excl[w][lane] = incl - len;
      if (lane == 31) s_excl[w][32] = total;
      __syncwarp();
      int n_ang = 0, n_ro = 0;  // this species: angular entries, radial-only entries
      for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        bool is_a = false, is_ro = false;
        int entry = 0;
        if (t < total) {
          int lo = 0, hi = 26;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_excl[w][mid] <= t) lo = mid; else hi = mid - 1;
          }
          const int j = s_start[w][lo] + (t - s_excl[w][lo]);
          const float4 pj = ws.pos4[j];
          const float dx = (pj.x - pi.x) + (float)(lo / 9 - 1) * ell[0];
          const float dy = (pj.y - pi.y) + (float)((lo / 3) % 3 - 1) * ell[1];
          const float dz = (pj.z - pi.z) + (float)(lo % 3 - 1) * ell[2];
          const float r2 = dx * dx + dy * dy + dz * dz;
          const bool is_r = r2 < rcr2 && !(j == row && lo == 13);
          is_a = is_r && r2 < rca2;
          is_ro = is_r && !is_a;
          entry = pack_nbr(j, lo);
        }
        const unsigned ba = __ballot_sync(0xffffffffu, is_a);
        const unsigned bro = __ballot_sync(0xffffffffu, is_ro);
        const unsigned below = (1u << lane) - 1u;
        if (is_a) {
          const int pos = nr + n_ang + __popc(ba & below);
          if (pos < ws.cap_r) lr[pos] = entry;
        }
        if (is_ro) {
          const int pos = n_ro + __popc(bro & below);
          if (pos < ws.cap_r) stage[pos] = entry;
        }
        n_ang += __popc(ba);
        n_ro += __popc(bro);
      }
      __syncwarp();
      // append the radial-only entries after this species' angular ones
      const int base = nr + n_ang;
      for (int k = lane; k < n_ro; k += 32)
        if (base + k < ws.cap_r && k < ws.cap_r) lr[base + k] = stage[k];
      __syncwarp();
      // counts clamped to what the list holds, so readers never run past it
      const int keep = max(0, min(n_ang + n_ro, ws.cap_r - nr));
      const int keep_a = min(n_ang, keep);
      if (lane == 0) { cr[sp] = keep; ca[sp] = keep_a; }
      nr += n_ang + n_ro;
      na += n_ang;
    }
    if (lane == 0) {
      for (int sp = P.S; sp < kMaxS; ++sp) { cr[sp] = 0; ca[sp] = 0; }
      atomicMax(&ws.flags[kFlagMaxNbrR], nr);
      atomicMax(&ws.flags[kFlagMaxNbrA], na);
      if (nr > ws.cap_r) atomicOr(&ws.flags[kFlagOverflowR], 1);
      if (na > ws.cap_a) atomicOr(&ws.flags[kFlagOverflowA], 1);
    }
  }
}

size_t neighbors_smem(int cap_r) { return 8 * sizeof(int) * (size_t)cap_r; }

cudaError_t neighbors_set_smem_limits() {
  return cudaFuncSetAttribute(k_neighbors, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)neighbors_smem(4096));
}

}  // namespace nnp
