#include "plan.h"

#include <algorithm>
#include <cmath>

#include "morph_geom.h"

namespace morph {

namespace {
Tuning g_tuning;
bool g_init = false;
}  // namespace

// Estimated time of one launch configuration (arbitrary units): each phase
// of a tile costs (rounds of 128 threads over its work items) x (work per
// item); tiles run in waves of (152 SMs x CTAs per SM).  Only used to rank
// tile shapes; the autotuner measures the classes it is asked about.
int ctas_per_sm(int smem_bytes);

double tile_cost(const FusedLaunch& L, int cfg) {
  const int TX = tile_tx(cfg), TY = tile_ty(cfg);
  const Geom g = make_geom(L.esz, TX, TY, L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row);
  if (g.smem_bytes > kMaxSmemBytes) return 1e30;
  const double thr = 128.0;
  auto rounds = [&](double items) { return std::ceil(items / thr); };
  const double nk = g.noct - g.k0, ntc = TY / 8.0, nxo = TX / 8.0;
  double t = 4.0 + rounds(g.ih * g.noct * 2.0 * L.esz / 4.0) * 0.5;  // landing, fix-up
  if (L.wy > 1) {
    if (L.vhgw_col)
      t += rounds(nk * g.nchy) * 10.0 + rounds(nk * ntc) * (20.0 + L.wy / 8.0);
    else
      t += rounds(nk * ntc) * (8.0 + L.wy) * 1.2;
  } else if (L.wx > 1) {
    t += rounds(nk * ntc) * 10.0;
  }
  if (L.wx > 1) {
    if (L.vhgw_row)
      t += rounds(ntc * g.nchx) * 10.0 + rounds(nxo * ntc) * (28.0 + L.wx / 8.0);
    else
      t += rounds(nxo * ntc) * ((8.0 + L.wx) * 1.2 + 8.0);
  }
  const int per_sm = ctas_per_sm(g.smem_bytes);
  const double ntiles = std::ceil(static_cast<double>(L.W) / TX) * std::ceil(static_cast<double>(L.H) / TY);
  const double slots = 152.0 * per_sm;
  const double waves = std::ceil(ntiles / slots);
  // A CTA is 4 warps: with fewer than 3 CTAs on an SM its barriers and loads
  // leave the issue slots idle (measured: 1 CTA/SM ran at 6% active warps).
  const double occ = per_sm >= 3 ? 1.0 : per_sm == 2 ? 1.35 : 2.2;
  return waves * t * occ * (ntiles < slots ? 1.0 : per_sm) / per_sm;
}

int ctas_per_sm(int smem_bytes) {
  int per_sm = 232448 / (smem_bytes + 1024);  // shared memory per SM / per CTA
  if (per_sm > 4) per_sm = 4;                 // registers: 4 CTAs of 128 threads
  return per_sm < 1 ? 1 : per_sm;
}

bool plan_split(const FusedLaunch& L) {
  const Tuning& t = tuning();
  if (L.wx <= 1 || L.wy <= 1) return false;
  if (t.split_mode == 0) return false;
  if (t.split_mode == 1) return true;
  // auto: two launches when both passes take the van Herk/Gil-Werman method
  // (above the crossovers), i.e. run on the single-pass kernels, which then
  // pay for the second trip through memory (the intermediate mostly stays
  // in L2).  Measured on the GB300 at 4096^2 (CUDA-graph timing): 9 x 9 to
  // 21 x 21 with both passes by van Herk/Gil-Werman take 19.4-20.8 us (u8)
  // and 24.2-25.0 us (u16) as two launches against 29.7-32.0 and 33.2-38.2
  // fused, and 127 x 127 runs about 3x faster; with a direct-method pass (3
  // x 3 to 9 x 9 at a crossover of 9) the fused kernel was 7-39% faster.  Below 2 Mpixels the second launch's
  // fixed cost is not repaid, and the fused kernel is kept.  Also whenever
  // the fused tile the planner picks (or every fused tile) would run fewer
  // than 3 CTAs per SM.  A window with one pass by van Herk/Gil-Werman
  // and the other direct splits from 4 Mpixels (the direct pass then runs
  // on the row or column kernel): measured at 4096^2, u8 5 x 40 38.3 ->
  // 22.6 us, 40 x 5 33.0 -> 24.0 us (u16 41.5 -> 37.9, 35.1 -> 28.3); at
  // 2048^2 12.9 -> 9.7 and 11.4 -> 9.3 (u16 15.4 -> 15.0, 14.9 -> 11.9);
  // at 1448^2 the fused kernel was still up to 30% faster.
  const int e = L.esz - 1;
  const bool vhgw_y = L.wy > t.cross_col[e] && L.wy >= 8, vhgw_x = L.wx > t.cross_row[e] && L.wx >= 8;
  const long long px = static_cast<long long>(L.W) * L.H;
  if (px >= (2ll << 20) && vhgw_x && vhgw_y) return true;
  if (px >= (4ll << 20) && (vhgw_x || vhgw_y)) return true;
  FusedLaunch F = L;
  if (!plan_single(&F)) return true;
  return ctas_per_sm(fused_smem_bytes(F)) < 3;
}

void reset_tuning_defaults() {
  for (int e = 0; e < 2; ++e) {
    g_tuning.cross_col[e] = 9;
    g_tuning.cross_row[e] = 9;
    g_tuning.forced_cfg[e] = -1;
    g_tuning.xpass_transpose[e] = 0;
  }
  g_tuning.split_mode = -1;
  g_tuning.batch_alone = kBatchAlonePixels;
  g_tuning.comp_mode = -1;
  g_tuning.split_order = 1;
  g_tuning.pdl_mode = 1;
  g_tuning.pipe_mode = -1;
  g_tuning.col_mode = -1;
  g_tuning.row_mode = -1;
  g_tuning.colv_mode = -1;
  g_tuning.colv_rows = 0;
  g_tuning.colv_lb = 0;
  g_tuning.rowv_mode = -1;
  g_tuning.rowv_seg = 0;
  g_tuning.rowv_rr[0] = g_tuning.rowv_rr[1] = 0;
  for (int e = 0; e < 2; ++e) {
    for (int c = 0; c < 4; ++c) g_tuning.fused_cfg_tuned[e][c][0] = g_tuning.fused_cfg_tuned[e][c][1] = -1;
    for (int c = 0; c < 5; ++c) g_tuning.colv_fam_tuned[e][c] = -1;
  }
  g_tuning.from_autotune = 0;
  g_init = true;
}

int fused_tune_class(int wx, int wy) {
  const int m = wx > wy ? wx : wy;
  return m <= 3 ? 0 : m <= 5 ? 1 : m <= 7 ? 2 : m <= 9 ? 3 : -1;
}

int colv_tune_class(int wy) { return wy <= 24 ? 0 : wy <= 40 ? 1 : wy <= 76 ? 2 : wy <= 114 ? 3 : 4; }

int colv_family_rows(int fam, int wy) {
  switch (fam) {
    case 1: return wy;
    case 2: return 2 * wy;
    case 3: return 3 * wy;
    case 4: return 64;
    case 5: return 128;
    case 6: return 256;
  }
  return 0;  // the built-in rule
}

Tuning& tuning() {
  if (!g_init) reset_tuning_defaults();
  return g_tuning;
}

// Persistent prefetching form: when its layout fits and (auto) the window is
// 1 x wy and the image has at least two tiles per resident CTA of it.  On
// the GB300 the doubled input buffer costs a resident CTA per SM; only the
// single pass along y gained from the overlap (measured: up to 15%), windows
// with a pass along x lost up to 40%.
void set_pipe(FusedLaunch* L) {
  const Tuning& t = tuning();
  L->pipe = false;
  if (t.pipe_mode == 0) return;
  const int b = fused_pipe_smem_bytes(*L);
  if (b <= 0 || b > kMaxSmemBytes) return;
  if (t.pipe_mode == 1) {
    L->pipe = true;
    return;
  }
  if (L->wx != 1 || L->wy == 1) return;
  const double ntiles = std::ceil(static_cast<double>(L->W) / tile_tx(L->cfg)) *
                        std::ceil(static_cast<double>(L->H) / tile_ty(L->cfg));
  L->pipe = ntiles >= 2.0 * 152 * ctas_per_sm(b);
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
    if (b > 0 && b <= kMaxSmemBytes) {
      set_pipe(L);
      return true;
    }
  }
  // the tile shape the autotuner measured for this pixel type, window
  // class and size class (direct-method windows on images of at least
  // 1 Mpixel)
  const int fc = fused_tune_class(L->wx, L->wy);
  const long long px = static_cast<long long>(L->W) * L->H;
  const int sc = fused_size_class(px);
  if (fc >= 0 && !L->vhgw_col && !L->vhgw_row && px >= (1ll << 20) && t.fused_cfg_tuned[e][fc][sc] >= 0) {
    L->cfg = t.fused_cfg_tuned[e][fc][sc];
    const int b = fused_smem_bytes(*L);
    if (b > 0 && b <= kMaxSmemBytes) {
      set_pipe(L);
      return true;
    }
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
  set_pipe(L);
  return true;
}

}  // namespace morph
