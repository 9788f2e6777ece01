// Method and tile choice for one launch (section 5.3's final combination:
// the direct method up to a crossover window, van Herk/Gil-Werman above it;
// the crossovers are set per pixel type and axis, by default or by the
// autotuner measuring this GPU).
#pragma once

#include "morph_internal.h"

namespace morph {

struct Tuning {
  int cross_col[2];  // [esz-1]: pass along y uses the direct method iff wy <= cross_col
  int cross_row[2];  // [esz-1]: pass along x uses the direct method iff wx <= cross_row
  int forced_cfg[2];              // [esz-1]: tile configuration to use when it fits (-1: cost model)
  int from_autotune;              // 1 once measured or loaded from a cache
};

Tuning& tuning();
void reset_tuning_defaults();

// Fills L->vhgw_col, L->vhgw_row and L->cfg; false if no tile configuration
// fits the window in shared memory.
bool plan_single(FusedLaunch* L);

}  // namespace morph
