#include "plan.h"

#include <cmath>

#include "morph_geom.h"

namespace morph {

namespace {
Tuning g_tuning;
bool g_init = false;

// Relative cost of one launch configuration per output pixel, from the work
// each phase does on the tile (input area for the load and the y pass, the
// x pass on the y-pass output, two transposes) and a penalty for low
// occupancy.  Only used to rank tile shapes; the autotuner can override.
double tile_cost(const FusedLaunch& L, int cfg) {
  const double TX = tile_tx(cfg), TY = tile_ty(cfg);
  const Geom g = make_geom(L.esz, tile_tx(cfg), tile_ty(cfg), L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row);
  if (g.smem_bytes > kMaxSmemBytes) return 1e30;
  const double iw = 8.0 * (g.noct - g.k0), ih = g.ih;
  double cost = iw * ih / (TX * TY) * 0.5;  // TMA landing, border fix-up
  if (L.wy > 1) {
    // y pass per output octet: blocked = scan of (ih/TY) inputs + combine,
    // direct = (w+7)/8 row reads per output
    const double per = L.vhgw_col ? 2.0 * ih / TY + 2.0 + L.wy / 64.0 : (L.wy + 7.0) / 8.0 + 1.0;
    cost += iw / TX * per;
  }
  if (L.wx > 1) {
    const double xin = (TX + L.wx - 1) / TX;
    const double per = L.vhgw_row ? 2.0 * xin + 2.0 + L.wx / 64.0 : (L.wx + 7.0) / 8.0 + 1.0;
    cost += 1.0 * iw / TX + 1.0 + per;  // transposes + the pass
  }
  // CTAs per SM from shared memory and from registers (2 CTAs of 256 threads)
  int per_sm = (232448) / (g.smem_bytes + 1024);
  if (per_sm > 2) per_sm = 2;
  if (per_sm < 1) per_sm = 1;
  cost *= per_sm >= 2 ? 1.0 : 1.4;
  // few CTAs for a small image: the GPU (152 SMs) is not filled
  const double ctas = std::ceil(L.W / TX) * std::ceil(L.H / TY);
  if (ctas < 152.0 * per_sm) cost *= 1.0 + 0.5 * (1.0 - ctas / (152.0 * per_sm));
  return cost;
}
}  // namespace

void reset_tuning_defaults() {
  for (int e = 0; e < 2; ++e) {
    g_tuning.cross_col[e] = 9;
    g_tuning.cross_row[e] = 9;
    g_tuning.forced_cfg[e] = -1;
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
  // The blocked large-window method needs windows of at least 8 (its block).
  L->vhgw_col = L->wy > t.cross_col[e] && L->wy >= 8;
  L->vhgw_row = L->wx > t.cross_row[e] && L->wx >= 8;
  if (t.forced_cfg[e] >= 0) {
    L->cfg = t.forced_cfg[e];
    const int b = fused_smem_bytes(*L);
    if (b > 0 && b <= kMaxSmemBytes) return true;
  }
  double best = 1e29;
  int best_cfg = -1;
  for (int c = 0; c < kNumTileCfg; ++c) {
    const double v = tile_cost(*L, c);
    if (v < best) {
      best = v;
      best_cfg = c;
    }
  }
  if (best_cfg < 0) return false;
  L->cfg = best_cfg;
  return true;
}

}  // namespace morph
