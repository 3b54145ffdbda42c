// The layout table: which kernel layout the launchers use for a (routine,
// order, batch size) when a caller -- the autotuner -- has chosen one
// (bf_layout_set), instead of the built-in rule.  Host code only.
//
// The paper's library comes in size-specialized variants chosen at build
// time for the target (Sec. 5.1: HP2, HP2F); here the variants are kernel
// layouts (problems per CTA, lanes per problem, split of the k-loop), and the
// choice is made per problem size at run time.
#include <atomic>

#include "bf_internal.cuh"

namespace bf {
namespace {

constexpr int KEY_N = 513;        // orders 0..511, and one slot for every larger order
constexpr int KEY_BATCH = 32;     // batch sizes by floor(log2(batch))
std::atomic<signed char> g_table[ROUTINE_COUNT][KEY_N][KEY_BATCH];

inline int key_n(int n) { return n < KEY_N - 1 ? (n < 0 ? 0 : n) : KEY_N - 1; }
inline int key_batch(int batch) {
  int k = 0;
  while (k < KEY_BATCH - 1 && (2LL << k) <= (long long)batch) k++;
  return k;
}

int layout_count(int routine) {
  switch (routine) {
    case ROUTINE_GEMM_NT: case ROUTINE_SYRK_LN: return LAYOUT_GEMM_COUNT;
    case ROUTINE_POTRF: case ROUTINE_SYRK_POTRF: return LAYOUT_CHOL_COUNT;
    case ROUTINE_TRSM_RLTN: return LAYOUT_TRSM_COUNT;
    case ROUTINE_GETRF: return LAYOUT_LU_COUNT;
    case ROUTINE_GELQF: return LAYOUT_LQ_COUNT;
    default: return 0;
  }
}

bool layout_ok(int routine, int layout, int n) {
  switch (routine) {
    case ROUTINE_GEMM_NT: case ROUTINE_SYRK_LN: return layout >= 1 && layout < LAYOUT_GEMM_COUNT;
    case ROUTINE_POTRF: case ROUTINE_SYRK_POTRF: return chol_layout_ok(layout, n);
    case ROUTINE_TRSM_RLTN: return trsm_layout_ok(layout, n);
    case ROUTINE_GETRF: return getrf_layout_ok(layout, n);
    // keyed by the column count n; the row count is checked at the call
    case ROUTINE_GELQF: return gelqf_layout_ok(layout, 1, n);
    default: return false;
  }
}

}  // namespace

int layout_forced(int routine, int n, int batch) {
  if (routine < 0 || routine >= ROUTINE_COUNT) return 0;
  return g_table[routine][key_n(n)][key_batch(batch)].load(std::memory_order_relaxed);
}

}  // namespace bf

using namespace bf;

extern "C" {

int bf_layout_count(int routine) { return layout_count(routine); }

int bf_layout_set(int routine, int n, int batch, int layout) {
  if (routine < 0 || routine >= ROUTINE_COUNT) return -1;
  if (n < 0) return -2;
  if (batch < 1) return -3;
  if (layout < 0 || layout >= layout_count(routine)) return -4;
  if (layout != 0 && !layout_ok(routine, layout, n)) return BF_ERR_UNSUPPORTED;
  g_table[routine][key_n(n)][key_batch(batch)].store((signed char)layout, std::memory_order_relaxed);
  return 0;
}

int bf_layout_get(int routine, int batch, int m, int n, int k) {
  if (routine < 0 || routine >= ROUTINE_COUNT) return -1;
  if (batch < 1) return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  const int order = (routine == ROUTINE_TRSM_RLTN || routine == ROUTINE_GELQF) ? n : m;
  const int forced = layout_forced(routine, order, batch);
  if (forced > 0 && (routine != ROUTINE_GELQF || gelqf_layout_ok(forced, m, n))) return forced;
  switch (routine) {
    case ROUTINE_GEMM_NT: return gemm_layout_rule(false, batch, m, n, k);
    case ROUTINE_SYRK_LN: return gemm_layout_rule(true, batch, m, m, k);
    case ROUTINE_POTRF: return chol_layout_rule(false, batch, m);
    case ROUTINE_SYRK_POTRF: return chol_layout_rule(true, batch, m);
    case ROUTINE_GETRF: return getrf_layout_rule(batch, m);
    case ROUTINE_GELQF: return gelqf_layout_rule(batch, m, n);
    default: return trsm_layout_rule(batch, m, n);
  }
}

void bf_layout_reset(void) {
  for (int r = 0; r < ROUTINE_COUNT; r++)
    for (int i = 0; i < KEY_N; i++)
      for (int j = 0; j < KEY_BATCH; j++) g_table[r][i][j].store(0, std::memory_order_relaxed);
}

}  // extern "C"
