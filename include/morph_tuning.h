/*
 * morph_tuning.h -- tuning and test hooks of the GB300 morphology library.
 *
 * Each switch below forces one kernel, launch form or scheduling choice of
 * the single-image calls of morph.h, for the parity tests (every kernel is
 * checked on its own against the CPU oracle), for profiling one kernel, and
 * for the measurements that set the library's defaults.  None of them
 * changes a result: every kernel computes the exact section 2 definition.
 * The settings are process-wide (not per device or thread) and take effect
 * for calls made after them; morph_reset_tuning (morph.h) restores every
 * default.  Each returns MORPH_OK, or MORPH_ERR_ARG (MORPH_ERR_DTYPE for a
 * bad dtype) for a value it does not accept.
 */
#ifndef MORPH_TUNING_H
#define MORPH_TUNING_H

#include "morph.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Form of single-image calls with a 2-D window (section 5: the element is
 * separable, so erosion by wx x wy is erosion by 1 x wy followed by wx x 1).
 * mode -1 (default): two launches through an intermediate image the
 * library allocates stream-ordered for images of at least 2 Mpixels when
 * both passes take the van Herk/Gil-Werman method (both window sides above
 * the crossovers of morph_set_tuning; there the single-pass kernels were
 * measured faster than the fused kernel on the GB300), for images of at
 * least 4 Mpixels when one pass takes that method and the other the direct
 * one (the direct pass then runs on the row or column kernel), or when the
 * fused tile is so large that fewer than 3 CTAs fit on an SM; otherwise
 * both passes fused in one kernel.  0: always fused; 1: always two
 * launches.  The result never changes.
 */
int morph_set_split(int mode);

/*
 * Order of the two launches of that form (section 5: the passes commute):
 * 1 (default) the pass along x first, 0 the pass along y first.  On the
 * GB300 the pass along x first was measured 6-13% faster (at 4096^2, 15 x 15
 * to 127 x 127): the pass along y then reads the intermediate image while it
 * is still in L2.  The result never changes.  MORPH_ERR_ARG for another
 * order.
 */
int morph_set_split_order(int order);

/*
 * Whether the kernels of single-image calls are launched with programmatic
 * stream serialisation (1) or not (0).  With it a kernel may be scheduled
 * while the previous kernel on its stream drains: that kernel lets its
 * successor in once each of its CTAs has finished its work, and the
 * successor's CTAs wait (griddepcontrol.wait) for the predecessor to finish
 * and flush its memory before touching global memory, so the launch gap
 * between consecutive calls overlaps the previous call's tail.  On by
 * default: on the GB300 at 4096^2 it made single-stream calls 0-4% faster
 * and two streams of independent calls 2% faster.  A GPU scheduling
 * choice; the result never changes.  MORPH_ERR_ARG for another value.
 */
int morph_set_pdl(int on);

/*
 * Launch form of the fused kernel for single-image calls (no counterpart in
 * the paper: a GPU scheduling choice).  mode 1: a persistent grid (resident
 * CTAs x SMs) whose CTAs walk the tiles in turn, with two input buffers per
 * CTA so that the TMA load of a CTA's next tile overlaps the computation of
 * its current one; 0: one CTA per tile; -1 (default): the persistent form
 * when the image has at least two tiles per resident CTA and its doubled
 * input buffer fits in shared memory.  Images whose rows are not 16-byte
 * aligned always take one CTA per tile.  The result never changes.
 * Returns MORPH_ERR_ARG for another mode.
 */
int morph_set_pipeline(int mode);

/*
 * Kernel for single-image calls whose window is 1 x wy (wy > 1), including
 * the first launch of the two-launch form: mode -1 (default) or 1: the
 * column kernel (one pass along y per CTA tile 128 bytes wide and as tall as
 * fills whole waves of the GPU; outputs stored from registers); 0: the
 * fused two-pass tile kernel.  The result never changes.  MORPH_ERR_ARG for
 * another mode.
 */
int morph_set_column_kernel(int mode);

/*
 * Kernel of the pass along y (1 x wy windows, and the first launch of the
 * two-launch form): van Herk/Gil-Werman with blocks of wy rows (section
 * 5.1.1), one warp per strip of 32 lanes x lane_bytes bytes and `rows`
 * output rows, the block suffix kept in place of the input rows it
 * replaces.  mode 1: this kernel for every wy >= 2 whose warp tile fits in
 * shared memory; -1 (default): wherever the van Herk/Gil-Werman method is
 * chosen (wy above the crossover of section 5.3; measured faster than the
 * column kernel there); 0: never (the column kernel of
 * morph_set_column_kernel instead).  rows: output rows per warp tile, 1 to
 * 1024, or 0 for the measured default (a multiple of wy filling one or two
 * 32-row input boxes below 32 rows; else wy or 2 wy up to 256, or 64, with
 * 64 or 32 where those tiles would leave the GPU's SMs short of warps).
 * lane_bytes: 4 (strips 128 bytes wide), 8 (256 bytes, two independent scan
 * chains per lane), or 0 for the built-in rule.  The result never changes.  MORPH_ERR_ARG for another
 * mode, rows or lane_bytes.
 */
int morph_set_colv(int mode, int rows, int lane_bytes);

/*
 * Kernel of the pass along x (wx x 1 windows, and the second launch of the
 * two-launch form): van Herk/Gil-Werman with blocks of 8 pixels (section
 * 5.1.1's decomposition; the whole blocks inside a window folded from their
 * totals), one warp per 2 (default), 4 or 8 rows and a segment of `seg`
 * output columns, each lane's block transposed in registers (section 4) so
 * that one packed min/max handles 2 rows.  Accepts 9 <= wx <= 256 when the
 * source rows are aligned to 8 bytes (u8) or 16 bytes (u16).  mode 1: this
 * kernel wherever it accepts the call; 2, 3 and 4: the same with 8, 4 and 2
 * rows per warp; -1 (default): wherever the van Herk/Gil-Werman method is
 * chosen (measured faster than the row kernel of morph_set_row_kernel
 * there); 0: never.  seg: output columns per warp task,
 * rounded up to a multiple of 256, or 0 for the shortest segment whose
 * tasks fit in one wave of resident warps.  The result never changes.
 * MORPH_ERR_ARG for another mode or seg.
 */
int morph_set_rowv(int mode, int seg);

/*
 * Kernel for single-image calls whose window is wx x 1 (wx > 1), including
 * the second launch of the two-launch form: mode -1 (default) or 1: the row
 * kernel (tiles 256 bytes wide; 8 x 8-pixel blocks transposed once in
 * registers into a column-major shared-memory copy, the pass along x run on
 * it, outputs transposed back and stored from registers) when its tile fits
 * in shared memory; 0: the fused two-pass tile kernel.  The result never
 * changes.  MORPH_ERR_ARG for another mode.
 */
int morph_set_row_kernel(int mode);

/*
 * Form of the pass along x for dtype (MORPH_U8/MORPH_U16).  mode 0 (default):
 * inside the fused kernel, whose 8x8-pixel register transposes turn it into a
 * pass along y (section 1's "transpose, pass, transpose" without leaving the
 * chip); 1: the paper's baseline form of section 5.2.1 through HBM --
 * transpose_u8/u16 into a scratch image, the pass along y, transpose back --
 * with a 2-D window's 1 x wy pass run first.  Scratch images come from the
 * stream-ordered allocator.  morph_autotune measures both and keeps the
 * faster.  The result never changes.  MORPH_ERR_DTYPE / MORPH_ERR_ARG for a
 * bad dtype or mode.
 */
int morph_set_xpass(int dtype, int mode);

/*
 * Images of morph_batch and morph_batch_plan_create with at least
 * min_pixels pixels run as their single call (morph_apply's launches, on the
 * batch's stream after the batched launches), besides those that always do
 * (see morph_batch); the rest share the batched launches.  0 (the default):
 * no size rule; negative: the default.  The result never changes.  Returns
 * MORPH_OK.
 */
int morph_set_batch_alone(long long min_pixels);

/*
 * Form of morph_composite.  The one-pass kernel (windows of at most 9 x 9
 * pixels, on images at least as large as the window) loads each output tile
 * with the halo of both steps and runs all of their 1-D passes (the
 * gradient's min and max side by side) in shared memory, so each pixel
 * crosses HBM once in and once out; the other form is two ordinary calls
 * through an intermediate image (and, for the gradient, a subtraction pass).
 * -1 (auto, the default): the one-pass kernel for the gradient of windows up
 * to 5 x 5, where it measured faster; 1: the one-pass kernel wherever it
 * fits; 0: never.  The result never changes.  MORPH_ERR_ARG for another
 * value.
 */
int morph_set_composite_kernel(int mode);

#ifdef __cplusplus
}
#endif

#endif /* MORPH_TUNING_H */
