// nnp_tune.cu -- launch-shape autotuner (NNP_FLAG_AUTOTUNE).
//
// The neighbour, descriptor and descriptor-backward kernels are persistent:
// a grid capped at (blocks per SM) x SMs.  The warps of the first two take
// their work items -- cells, tiles of consecutive row pairs -- in static
// order or from a queue; the backward's warps take rows in static order.  The
// neighbour kernel can also split each cell's row groups over two warps.  The best cap and tile depend
// on the row count and on how many systems share the launch (a batch of many
// small boxes has other tails and another locality than one large box).  On
// the first synchronous evaluation of a (species, precision, row-count
// bucket, batch or single) the tuner runs the pipeline directly (no graph)
// over eight candidate shapes per kernel, evaluated side by side (candidate
// i of every kernel in the same run), times each stage with CUDA events (three
// repetitions after a warm-up), keeps the fastest shape per stage, and caches
// it in memory and, if the environment variable NNP_AUTOTUNE_CACHE names a
// file, in that file ("key nbr fwd bwd fwd_tile bwd_tile nbr_queue" lines)
// for later processes.  The static shapes are among the candidates, and a
// queue shape is kept only where it measures at least 3% faster than the
// best static one.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>

#include "nnp_host.h"

namespace {
std::mutex g_mu;
std::map<long long, nnp_ctx::Tune> g_cache;
bool g_file_loaded = false;

void load_file() {
  if (g_file_loaded) return;
  g_file_loaded = true;
  const char* path = std::getenv("NNP_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  long long key;
  nnp_ctx::Tune t;
  while (std::fscanf(f, "%lld %d %d %d %d %d %d", &key, &t.nbr, &t.fwd, &t.bwd, &t.fwd_tile, &t.bwd_tile,
                     &t.nbr_dyn) == 7)
    if (t.nbr > 0 && t.fwd > 0 && t.bwd > 0 && t.fwd_tile != 0 && t.bwd_tile != 0) g_cache[key] = t;
  std::fclose(f);
}

void save_entry(long long key, const nnp_ctx::Tune& t) {
  const char* path = std::getenv("NNP_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%lld %d %d %d %d %d %d\n", key, t.nbr, t.fwd, t.bwd, t.fwd_tile, t.bwd_tile, t.nbr_dyn);
  std::fclose(f);
}
}  // namespace

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

int nnp_ctx::autotune(long long n, int B, long long bins, long long rows) {
  const int bucket = (int)std::ceil(std::log2((double)(rows > 2 ? rows : 2)));
  const long long key = ((long long)P.S * 4 + cfg.precision) * 64 + bucket + (B > 1 ? 1000000 : 0);
  if (key == tuned_key) return NNP_OK;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    load_file();
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      tune = it->second;
      tuned_key = key;
      invalidate_graph();
      return NNP_OK;
    }
  }
  // candidates, column i of each list timed in the same pipeline run: the
  // neighbour kernel's (blocks per SM, form: bit 0 items from the queue, bit
  // 1 each cell's row groups over two warps), the descriptor kernels' (blocks
  // per SM, tile; tile < 0: static order).
  constexpr int kC = 8;
  const int cand_nbr[kC][2] = {{4, 0}, {8, 0}, {16, 0}, {16, 2}, {8, 1}, {16, 1}, {32, 1}, {16, 3}};
  const int cand_fwd[kC][2] = {{2, -1}, {4, -1}, {8, -1}, {16, -1}, {8, 1}, {8, 2}, {8, 4}, {16, 2}};
  const int cand_bwd[kC][2] = {{4, -1}, {8, -1}, {16, -1}, {32, -1}, {64, -1}, {12, -1}, {24, -1}, {48, -1}};
  const bool own_events = stage_ev[0] == nullptr;
  if (own_events)
    for (auto& ev : stage_ev) CK(cudaEventCreate(&ev));
  // fastest time per stage: [static shapes][queue shapes]
  float best[2][3] = {{1e30f, 1e30f, 1e30f}, {1e30f, 1e30f, 1e30f}};
  Tune st_best = tune, dy_best = tune;
  int rc = launch_pipeline(n, B, bins, rows);  // warm-up
  if (rc) return rc;
  for (int rep = 0; rep < 3 && !rc; ++rep)
    for (int i = 0; i < kC && !rc; ++i) {
      tune = Tune{cand_nbr[i][0], cand_fwd[i][0], cand_bwd[i][0], cand_fwd[i][1], cand_bwd[i][1], cand_nbr[i][1]};
      rc = launch_pipeline(n, B, bins, rows);
      if (rc) break;
      CK(cudaEventSynchronize(stage_ev[5]));
      float t_nbr = 0.f, t_fwd = 0.f, t_bwd = 0.f;
      CK(cudaEventElapsedTime(&t_nbr, stage_ev[1], stage_ev[2]));
      CK(cudaEventElapsedTime(&t_fwd, stage_ev[2], stage_ev[3]));
      CK(cudaEventElapsedTime(&t_bwd, stage_ev[4], stage_ev[5]));
      const int qn = cand_nbr[i][1] & 1, qf = cand_fwd[i][1] > 0, qb = cand_bwd[i][1] > 0;
      Tune& tn = qn ? dy_best : st_best;
      Tune& tf = qf ? dy_best : st_best;
      Tune& tb = qb ? dy_best : st_best;
      if (t_nbr < best[qn][0]) { best[qn][0] = t_nbr; tn.nbr = cand_nbr[i][0]; tn.nbr_dyn = cand_nbr[i][1]; }
      if (t_fwd < best[qf][1]) { best[qf][1] = t_fwd; tf.fwd = cand_fwd[i][0]; tf.fwd_tile = cand_fwd[i][1]; }
      if (t_bwd < best[qb][2]) { best[qb][2] = t_bwd; tb.bwd = cand_bwd[i][0]; tb.bwd_tile = cand_bwd[i][1]; }
    }
  // a queue shape replaces the best static one only if it is faster by more
  // than the tuner's own run-to-run spread (these runs are not graph
  // replays, and their caches are warm)
  constexpr float kQueueGain = 0.97f;
  Tune chosen = st_best;
  if (best[1][0] < kQueueGain * best[0][0]) { chosen.nbr = dy_best.nbr; chosen.nbr_dyn = dy_best.nbr_dyn; }
  if (best[1][1] < kQueueGain * best[0][1]) { chosen.fwd = dy_best.fwd; chosen.fwd_tile = dy_best.fwd_tile; }
  if (best[1][2] < kQueueGain * best[0][2]) { chosen.bwd = dy_best.bwd; chosen.bwd_tile = dy_best.bwd_tile; }
  if (own_events)
    for (auto& ev : stage_ev) {
      cudaEventDestroy(ev);
      ev = nullptr;
    }
  if (rc) return rc;
  tune = chosen;
  tuned_key = key;
  invalidate_graph();
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key] = chosen;
    save_entry(key, chosen);
  }
  return NNP_OK;
}
