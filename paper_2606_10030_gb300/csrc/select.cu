// Strategy selection hooks used by agg_groupby: the learned selector and the
// autotuner. (Filled in by mlp.cu / autotune.cu.)
#include "groupby.cuh"

namespace agg {

int select_learned(const float* feat, bool* ok) {
  (void)feat;
  *ok = false;
  return AGG_STRAT_GLOBAL;
}

agg_status autotune_pick(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops, const float* feat,
                         cudaStream_t s, int* strategy, int* smem_slots, int64_t* table_slots) {
  (void)keys; (void)vals; (void)n; (void)vdt; (void)s;
  *strategy = rule_strategy(feat, ops);
  *smem_slots = 0;
  *table_slots = 0;
  return AGG_OK;
}

}  // namespace agg
