#include "plan.h"

namespace morph {

namespace {
Tuning g_tuning;
bool g_init = false;
}  // namespace

void reset_tuning_defaults() {
  for (int e = 0; e < 2; ++e) {
    g_tuning.cross_col[e] = 11;
    g_tuning.cross_row[e] = 11;
    g_tuning.cfg_order[e][0] = kTile128x64;
    g_tuning.cfg_order[e][1] = kTile64x64;
    g_tuning.cfg_order[e][2] = kTile64x32;
    g_tuning.cfg_order[e][3] = kTile32x32;
  }
  g_tuning.from_autotune = 0;
  g_init = true;
}

Tuning& tuning() {
  if (!g_init) reset_tuning_defaults();
  return g_tuning;
}

bool plan_single(FusedLaunch* L) {
  Tuning& t = tuning();
  const int e = L->esz - 1;
  L->vhgw_col = L->wy > t.cross_col[e];
  L->vhgw_row = L->wx > t.cross_row[e];
  for (int i = 0; i < kNumTileCfg; ++i) {
    L->cfg = t.cfg_order[e][i];
    const int b = fused_smem_bytes(*L);
    if (b > 0 && b <= kMaxSmemBytes) return true;
  }
  return false;
}

}  // namespace morph
