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
  int split_mode;                 // 2-D windows as two 1-D launches: -1 auto, 0 never, 1 always
  int split_order;                // their order: 0 pass along y first, 1 (default) pass along x first
  int pdl_mode;                   // single-image launches with programmatic stream serialisation: 1 (default) or 0
  int pipe_mode;                  // persistent input-prefetching kernel: -1 auto, 0 never, 1 always
  int xpass_transpose[2];         // [esz-1]: pass along x through the transpose kernels (1) or fused (0)
  int col_mode;                   // 1 x wy windows by the column kernel: -1 auto (yes), 0 never, 1 always
  int row_mode;                   // wx x 1 windows by the row kernel: -1 auto (yes), 0 never, 1 always
  int colv_mode;                  // 1 x wy passes by the warp-tiled vHGW kernel: -1 auto, 0 never, 1 always
  int colv_rows;                  // its output rows per warp tile (0: launch-shape model)
  int colv_lb;                    // its bytes per lane (0: built-in rule; 4 or 8)
  int rowv_mode;                  // wx x 1 passes by the register-blocked vHGW kernel: -1 auto, 0 never, 1 always
  int rowv_seg;                   // its output columns per warp segment (0: launch-shape model)
  int rowv_rr[2];                 // [esz-1]: rows per warp of the pass along x (0: built-in, 2)
  int fused_cfg_tuned[2][4][2];   // [esz-1][window class][size class]: measured tile shape of the fused kernel, -1 none
  int colv_fam_tuned[2][5];       // [esz-1][window class]: measured tile-height choice of the pass along y, -1 none
  long long batch_alone;          // batch images of at least this many pixels run as their single call (0: none)
  int comp_mode;                  // composites by the one-pass kernel where it fits: -1 auto, 0 never, 1 always
  int from_autotune;              // 1 once measured or loaded from a cache
};

// Window classes of the measured fused tile shapes: the larger window side
// up to 3, 5, 7 or 9 (direct-method windows; -1 outside).
int fused_tune_class(int wx, int wy);
// Size classes of the measured fused tile shapes: images of 1 to 8 Mpixels
// (measured on 2048 x 2048), larger (measured on 4096 x 4096).
inline int fused_size_class(long long pixels) { return pixels >= (8ll << 20) ? 1 : 0; }
// Window classes of the measured tile heights of the pass along y: wy up to
// 24, 40, 76, 114, above (representatives 15, 31, 51, 101, 127).
int colv_tune_class(int wy);
// Tile-height choices the autotuner measures for the pass along y: 0 the
// built-in rule, 1..3 that many windows, 4..6 64, 128 or 256 rows.
constexpr int kColvFamilies = 7;
int colv_family_rows(int fam, int wy);

// Default of the size above which images of a batch run as their own
// single call: none (0).  Measured on the GB300 with 2000 images of 64 to
// 2048 pixels a side (128-byte pitched rows): every image in the batched
// launches 376 Gpixel/s, images of at least 2^20 pixels as single calls 253.
constexpr long long kBatchAlonePixels = 0;

Tuning& tuning();
void reset_tuning_defaults();

// Fills L->vhgw_col, L->vhgw_row and L->cfg; false if no tile configuration
// fits the window in shared memory.
bool plan_single(FusedLaunch* L);

// Whether a 2-D window runs as a 1 x wy launch into an intermediate image and
// a wx x 1 launch from it (auto: when the fused tile would run one CTA per
// SM).  Estimated cost of one tile configuration, CTAs per SM for a size.
bool plan_split(const FusedLaunch& L);
double tile_cost(const FusedLaunch& L, int cfg);
int ctas_per_sm(int smem_bytes);

// Runs one clipped single-image launch by the planned form (fused, two
// launches, or the pass along x through the transpose kernels); returns a
// morph_status.  Defined with the C ABI.
int launch_planned(FusedLaunch L, cudaStream_t stream);

}  // namespace morph
