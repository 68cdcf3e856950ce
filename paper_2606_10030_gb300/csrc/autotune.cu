// Autotuner: time the GROUP BY candidates on the actual query and
// cache the fastest by query signature. The exhaustive pick also labels the
// training data of the learned selector and measures its regret.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "groupby.cuh"

namespace agg {

struct TuneChoice {
  int strategy;
  int threads;
  int smem_slots;
  int items;  // rows a thread folds per iteration (4 or 8)
  int tile;   // rows per tile of a hash-partitioned build (0: from the column)
};

namespace {
std::mutex g_tmu;
using Sig = std::tuple<int, int, int, int, int, int>;
std::map<Sig, TuneChoice> g_cache;

Sig signature(int vdt, uint32_t ops, const float* f) {
  bool covered = false;
  const double est = distinct_estimate(f, &covered);
  return Sig(vdt, (int)ops, (int)std::lround(f[F_LOG2N]), (int)std::lround(std::log2(std::max(1.0, est))),
             (int)std::floor(f[F_TOP8] * 10.0f), f[F_ADJ_EQ] >= 0.5f ? 1 : 0);
}
}  // namespace

agg_status groupby_with(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                        const agg_options& o, cudaStream_t s, agg_groups** out, const float* known_feat,
                        double known_hll);

static int smem_slots_sized(const float* f, bool mm) {
  bool covered = false;
  const double est = distinct_estimate(f, &covered);
  const int maxs = mm ? 2048 : 4096;
  int64_t sl = next_pow2((int64_t)std::ceil(2.0 * est));
  if (sl < 256) sl = 256;
  if (sl > maxs) sl = maxs;
  return (int)sl;
}

static agg_status run_candidates(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                                 const float* feat, double hll, int reps, cudaStream_t s, agg_tune_result* r) {
  std::memset(r, 0, sizeof(*r));
  std::memcpy(r->features, feat, sizeof(float) * F_COUNT);
  const bool mm = ops_minmax(ops);
  const int sized = smem_slots_sized(feat, mm), maxs = mm ? 2048 : 4096;
  // axes: strategy; block size; shared table size; rows a thread folds per
  // iteration (4 or 8); tile of the hash-partitioned build (16 Ki rows or the
  // column-sized default; the build runs on tiles only when it partitions)
  TuneChoice c[AGG_TUNE_MAX];
  int nc = 0;
  c[nc++] = {AGG_STRAT_SMEM, 512, sized, 4, 0};
  if (maxs != sized) c[nc++] = {AGG_STRAT_SMEM, 512, maxs, 4, 0};
  c[nc++] = {AGG_STRAT_SMEM, 256, sized, 4, 0};
  c[nc++] = {AGG_STRAT_SMEM, 512, sized, 8, 0};
  c[nc++] = {AGG_STRAT_SMEM, 512, sized, 4, 16384};
  c[nc++] = {AGG_STRAT_GLOBAL, 256, 0, 4, 0};
  c[nc++] = {AGG_STRAT_GLOBAL, 512, 0, 8, 0};
  c[nc++] = {AGG_STRAT_SORT, 0, 0, 0, 0};
  cudaEvent_t a, b;
  AGG_CUDA_TRY(cudaEventCreate(&a));
  AGG_CUDA_TRY(cudaEventCreate(&b));
  for (int k = 0; k < 3; ++k) r->best_ms_per_strategy[k] = INFINITY;
  agg_status st = AGG_OK;
  // every candidate gets the global table size the sketch implies, so that
  // none of them pays for a second sketch of its own
  const int64_t tslots = table_slots_for(feat, n, hll);
  for (int i = 0; i < nc && st == AGG_OK; ++i) {
    agg_options o{};
    o.strategy = c[i].strategy;
    o.block_threads = c[i].threads;
    o.smem_slots = c[i].smem_slots;
    o.table_slots = c[i].strategy == AGG_STRAT_SORT ? 0 : tslots;
    o.items_per_thread = c[i].items;
    o.tile_rows = c[i].tile;
    float best = INFINITY;
    for (int rep = 0; rep < std::max(1, reps) && st == AGG_OK; ++rep) {
      agg_groups* g = nullptr;
      cudaEventRecord(a, s);
      st = groupby_with(keys, vals, n, vdt, ops, o, s, &g, feat, hll);
      cudaEventRecord(b, s);
      if (st != AGG_OK) break;
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      agg_groups_free(g);
      best = std::min(best, ms);
    }
    r->strategy[i] = c[i].strategy;
    r->threads[i] = c[i].threads;
    r->smem_slots[i] = c[i].smem_slots;
    r->items_per_thread[i] = c[i].items;
    r->tile_rows[i] = c[i].tile;
    r->ms[i] = best;
    const int k = c[i].strategy == AGG_STRAT_SMEM ? 0 : c[i].strategy == AGG_STRAT_GLOBAL ? 1 : 2;
    r->best_ms_per_strategy[k] = std::min(r->best_ms_per_strategy[k], best);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != AGG_OK) return st;
  r->ncand = nc;
  r->best = 0;
  for (int i = 1; i < nc; ++i)
    if (r->ms[i] < r->ms[r->best]) r->best = i;
  std::lock_guard<std::mutex> lk(g_tmu);
  g_cache[signature(vdt, ops, feat)] = c[r->best];
  return AGG_OK;
}

bool autotune_cached(int vdt, uint32_t ops, const float* feat, int* strategy, int* smem_slots) {
  std::lock_guard<std::mutex> lk(g_tmu);
  auto it = g_cache.find(signature(vdt, ops, feat));
  if (it == g_cache.end()) return false;
  *strategy = it->second.strategy;
  *smem_slots = it->second.smem_slots;
  return true;
}

agg_status autotune_pick(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                         const float* feat, double hll, cudaStream_t s, int* strategy, int* smem_slots,
                         int64_t* table_slots, int* items, int* tile_rows) {
  *table_slots = 0;
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    auto it = g_cache.find(signature(vdt, ops, feat));
    if (it != g_cache.end()) {
      *strategy = it->second.strategy;
      *smem_slots = it->second.smem_slots;
      *items = it->second.items;
      *tile_rows = it->second.tile;
      return AGG_OK;
    }
  }
  agg_tune_result r;
  agg_status st = run_candidates(keys, vals, n, vdt, ops, feat, hll, 1, s, &r);
  if (st != AGG_OK) return st;
  *strategy = r.strategy[r.best];
  *smem_slots = r.smem_slots[r.best];
  *items = r.items_per_thread[r.best];
  *tile_rows = r.tile_rows[r.best];
  return AGG_OK;
}

// Strategy chosen by the learned selector; defined with the MLP kernels.
int select_learned(const float* feat, bool* ok);

}  // namespace agg

using namespace agg;

extern "C" agg_status agg_autotune(const uint32_t* keys_dev, const void* vals_dev, int64_t n, agg_dtype vdtype,
                                   uint32_t ops, int reps, agg_tune_result* out, void* stream) {
  clear_error();
  AGG_CHECK_ARG(out != nullptr, "null result");
  AGG_CHECK_ARG(dtype_valid(vdtype), "invalid dtype");
  AGG_CHECK_ARG(ops != 0 && (ops & ~(uint32_t)AGG_ALL) == 0, "invalid ops");
  AGG_CHECK_ARG(n > 0 && n <= 0xFFFFFFFFll && keys_dev && vals_dev, "invalid column");
  cudaStream_t s = (cudaStream_t)stream;
  float feat[F_COUNT];
  agg_status st = sketch_features(keys_dev, n, vdtype, ops, 0, s, feat);
  if (st != AGG_OK) return st;
  double hll = 0.0;
  if (wants_hll(feat, n)) {
    st = hll_estimate(keys_dev, n, s, &hll);
    if (st != AGG_OK) return st;
  }
  return run_candidates(keys_dev, vals_dev, n, vdtype, ops, feat, hll, reps, s, out);
}

extern "C" int64_t agg_autotune_cache_size(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  return (int64_t)g_cache.size();
}

extern "C" void agg_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_cache.clear();
}

extern "C" agg_status agg_autotune_save(const char* path) {
  clear_error();
  AGG_CHECK_ARG(path != nullptr, "null path");
  FILE* f = std::fopen(path, "w");
  AGG_CHECK_ARG(f != nullptr, "cannot open %s", path);
  std::lock_guard<std::mutex> lk(g_tmu);
  std::fprintf(f,
               "# agg autotune cache: dtype ops log2n log2d top8dec sorted -> strategy threads smem_slots items "
               "tile_rows\n");
  for (const auto& kv : g_cache) {
    const Sig& k = kv.first;
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
                 std::get<3>(k), std::get<4>(k), std::get<5>(k), kv.second.strategy, kv.second.threads,
                 kv.second.smem_slots, kv.second.items, kv.second.tile);
  }
  std::fclose(f);
  return AGG_OK;
}

extern "C" agg_status agg_autotune_load(const char* path) {
  clear_error();
  AGG_CHECK_ARG(path != nullptr, "null path");
  FILE* f = std::fopen(path, "r");
  AGG_CHECK_ARG(f != nullptr, "cannot open %s", path);
  char line[256];
  std::lock_guard<std::mutex> lk(g_tmu);
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    int v[11];
    if (std::sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &v[7],
                    &v[8], &v[9], &v[10]) != 11)
      continue;
    if (v[6] < AGG_STRAT_SMEM || v[6] > AGG_STRAT_SORT) continue;
    if (v[9] != 0 && v[9] != 4 && v[9] != 8) continue;
    if (v[10] != 0 && (v[10] < 4096 || v[10] > 65536 || (v[10] & (v[10] - 1)) != 0)) continue;
    g_cache[Sig(v[0], v[1], v[2], v[3], v[4], v[5])] = TuneChoice{v[6], v[7], v[8], v[9], v[10]};
  }
  std::fclose(f);
  return AGG_OK;
}
