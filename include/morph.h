/*
 * morph.h -- C ABI of the GB300 (sm_103a) grayscale morphology library.
 *
 * Operation (paper, section 2, the erosion equation and the sentence after
 * it): for a source image S of width x height pixels and a rectangular
 * structuring element of wx x wy cells with anchor (anchor_x, anchor_y),
 *
 *   erosion   D(x,y) = min { S(x',y') : x' in [x-anchor_x, x-anchor_x+wx-1],
 *                                       y' in [y-anchor_y, y-anchor_y+wy-1] }
 *   dilation  D(x,y) = max { ... same window ... }
 *
 * where pixels outside the image are ignored (equivalently: padded with the
 * maximum value for erosion and with 0 for dilation).  The anchor counts from
 * the element's top-left cell; the conventional centre is floor(w/2).  The
 * paper's literal formula S(x - n + wx/2, ...), n in [0, wx-1], is the anchor
 * ceil(w/2)-1, which is the same cell for odd windows.
 *
 * The result is exact (integer min/max): every entry point gives the same
 * bytes as the definition, whatever kernel, tile shape or method it picks.
 * Computation is separable (section 5): a pass along x with a wx x 1 element
 * and a pass along y with a 1 x wy element, each by the direct ("linear")
 * method of sections 5.1.2/5.2.2 for small windows or by van Herk/Gil-Werman
 * (sections 5.1.1/5.2.1) for large ones, switched at a crossover window
 * (section 5.3) measured on this GPU.  Both passes run fused in one kernel.
 *
 * Conventions for every entry point below
 *  - Image pointers are DEVICE pointers (cudaMalloc / torch CUDA memory)
 *    unless the name ends in _host.  The caller owns all buffers.
 *  - Pitches are in bytes; pitch >= width * element size.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream) and return before the kernel finishes, except the
 *    _host entry point, which synchronises its stream.
 *  - Errors are returned as a negative morph_status; nothing is thrown
 *    across the ABI and no output is written when a call is rejected.
 *    A CUDA launch error maps to MORPH_ERR_CUDA.
 *  - src and dst must not overlap (MORPH_ERR_ALIAS): every tile reads a halo
 *    that neighbouring tiles write.
 *  - wx, wy >= 1; 0 <= anchor < w.  A window may be larger than the image
 *    (the window is clipped to the image).
 *  - Single-image calls allocate nothing, except the two-launch form of
 *    2-D windows (see morph_set_split) and the transpose form of the pass
 *    along x (see morph_set_xpass), which take their intermediate images
 *    from the stream-ordered allocator (cudaMallocAsync on the call's
 *    stream; such calls can be captured into a CUDA graph).
 */
#ifndef MORPH_H
#define MORPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MORPH_OK = 0,
    MORPH_ERR_NULL = -1,    /* a required pointer is NULL                     */
    MORPH_ERR_SIZE = -2,    /* width/height < 1 or too large                   */
    MORPH_ERR_WINDOW = -3,  /* wx or wy < 1, or beyond the supported maximum   */
    MORPH_ERR_ANCHOR = -4,  /* anchor outside [0, w)                           */
    MORPH_ERR_PITCH = -5,   /* pitch < width * element size, or a 16-bit image  
                               not 2-byte aligned (pointer or pitch)          */
    MORPH_ERR_ALIAS = -6,   /* source and destination buffers overlap          */
    MORPH_ERR_CUDA = -7,    /* a CUDA call failed (launch, copy, attribute)    */
    MORPH_ERR_NOMEM = -8,   /* a device/host allocation failed                 */
    MORPH_ERR_DTYPE = -9,   /* unknown dtype or op code                        */
    MORPH_ERR_ARG = -10,    /* any other invalid argument (count, plan, ...)   */
    MORPH_ERR_DEVICE = -11, /* a kernel reported an error in the device word   */
    MORPH_ERR_LIMIT = -12   /* more images than morph_batch_noalloc accepts    */
} morph_status;

/* dtype and op codes used by morph_apply and morph_desc. */
enum { MORPH_U8 = 0, MORPH_U16 = 1 };
enum { MORPH_ERODE = 0, MORPH_DILATE = 1 };

/* Largest window (after clipping to the image: a window never needs to be
 * longer than 2*side-1) that one fused launch accepts, per axis. */
#define MORPH_MAX_WINDOW 255

/*
 * Erosion / dilation of one 8-bit image (section 2; section 5 computes it on
 * 8-bit pixels).  src and dst are device buffers of height rows of `pitch`
 * bytes each (the same pitch for both).  Returns MORPH_OK or an error.
 */
int morph_erode(const uint8_t *src, int width, int height, size_t pitch,
                int wx, int wy, int anchor_x, int anchor_y,
                uint8_t *dst, void *stream);
int morph_dilate(const uint8_t *src, int width, int height, size_t pitch,
                 int wx, int wy, int anchor_x, int anchor_y,
                 uint8_t *dst, void *stream);

/* The same on 16-bit pixels (section 2 definition; identities 65535 / 0). */
int morph_erode_u16(const uint16_t *src, int width, int height, size_t pitch,
                    int wx, int wy, int anchor_x, int anchor_y,
                    uint16_t *dst, void *stream);
int morph_dilate_u16(const uint16_t *src, int width, int height, size_t pitch,
                     int wx, int wy, int anchor_x, int anchor_y,
                     uint16_t *dst, void *stream);

/*
 * General single-image form: separate source/destination pitches, dtype
 * (MORPH_U8 / MORPH_U16) and op (MORPH_ERODE / MORPH_DILATE) as codes.
 */
int morph_apply(const void *src, size_t src_pitch, void *dst, size_t dst_pitch,
                int width, int height, int dtype, int op,
                int wx, int wy, int anchor_x, int anchor_y, void *stream);

/*
 * Composite operations (section 2: opening, closing and the morphological
 * gradient are expressed through erosion, dilation and arithmetic), one call
 * on the caller's stream:
 *   MORPH_OPEN      dilation by the reflected element of the erosion:
 *                   dilate(erode(S, wx x wy, (ax, ay)), wx x wy,
 *                          (wx-1-ax, wy-1-ay)); idempotent for every window
 *   MORPH_CLOSE     erosion by the reflected element of the dilation
 *   MORPH_GRADIENT  dilate(S) - erode(S), both by the same element and
 *                   anchor (never negative)
 * Arguments as in morph_apply (kind replaces op; the anchor is the first
 * step's).  The library allocates one scratch image of width x height pixels
 * (pitch rounded to 16 bytes) with cudaMallocAsync on the stream and frees it
 * there, so the intermediate stays in L2 where it fits; the call is safe to
 * capture in a CUDA graph.  The gradient's subtraction is a separate
 * elementwise kernel.  Errors as morph_apply; MORPH_ERR_ARG for another kind,
 * MORPH_ERR_NOMEM when the scratch cannot be allocated.
 */
enum { MORPH_OPEN = 0, MORPH_CLOSE = 1, MORPH_GRADIENT = 2 };

/*
 * Asynchronous 2-D copy of `height` rows of `width_bytes` bytes between any
 * two of host (pinned for full speed and true asynchrony) and device memory,
 * in the order of `stream` (cudaMemcpy2DAsync with the direction taken from
 * the pointers).  No counterpart in the paper: the serving loop's host-copy
 * form stages request images through it.  MORPH_ERR_NULL for a null
 * pointer, MORPH_ERR_SIZE for height < 1, MORPH_ERR_PITCH when a pitch is
 * below width_bytes, MORPH_ERR_CUDA when the copy cannot be queued.
 */
int morph_copy_2d(void *dst, size_t dst_pitch, const void *src, size_t src_pitch,
                  size_t width_bytes, int height, void *stream);
int morph_composite(const void *src, size_t src_pitch, void *dst, size_t dst_pitch,
                    int width, int height, int dtype, int kind,
                    int wx, int wy, int anchor_x, int anchor_y, void *stream);

/*
 * Host-buffer form: src and dst are HOST pointers (pinned memory gives full
 * copy speed; pageable memory works).  The library copies the image to a
 * device staging buffer that it owns and reuses (grown on demand, one pair per
 * device, freed by morph_release_staging), filters it, copies the result
 * back and synchronises `stream` before returning.  Not thread-safe: calls
 * that share a device must not run concurrently.
 */
int morph_apply_host(const void *src, size_t src_pitch, void *dst, size_t dst_pitch,
                     int width, int height, int dtype, int op,
                     int wx, int wy, int anchor_x, int anchor_y, void *stream);
int morph_release_staging(void);

/*
 * Batched form (one launch over many independent images of different sizes,
 * windows and ops).  Each descriptor names one device image pair.
 */
typedef struct {
    const void *src;     /* device, width x height pixels, src_pitch bytes/row */
    void *dst;           /* device, same size, dst_pitch bytes per row         */
    int32_t width, height;
    int64_t src_pitch, dst_pitch;
    int16_t wx, wy, anchor_x, anchor_y;
    uint8_t op;          /* MORPH_ERODE or MORPH_DILATE */
    uint8_t dtype;       /* MORPH_U8 or MORPH_U16 */
    uint8_t pad[2];
} morph_desc;

/*
 * Runs all n images in one persistent kernel launch on `stream`.  The
 * descriptor array is on the host; the call copies it (and the derived tile
 * list) to device memory owned by the library, so descs may be reused as soon
 * as the call returns.  Asynchronous.
 */
int morph_batch(const morph_desc *descs_host, int n, void *stream);

/*
 * Host-buffer form for many images: descs[i].src and .dst are HOST pointers
 * (pinned memory lets the copies overlap the filtering; pageable memory
 * works but serialises), the other fields as for morph_batch.  The images
 * are filtered one after another through a pipeline the library owns per
 * device -- three device staging slots and three streams -- so that the copy
 * in of image i+1, the filtering of image i and the copy out of image i-1
 * run at the same time (the paper has no counterpart: it filters images in
 * host memory).  The work starts after what is queued on `stream`; the call
 * returns once every result is in host memory.  Staging memory is grown on
 * demand and kept until morph_release_staging.  Calls that share a device
 * are serialised.  Every descriptor is validated before anything is queued;
 * the first failing image's status is returned.
 */
int morph_apply_host_batch(const morph_desc *descs, int n, void *stream);

/*
 * Graph form of morph_batch: plan_create validates the descriptors, builds the
 * tile list in device memory at fixed addresses and captures the persistent
 * launch in a CUDA graph; plan_launch replays it on `stream` (one
 * cudaGraphLaunch).  The image buffers must stay alive and at the same
 * addresses until plan_destroy.
 */
int morph_batch_plan_create(const morph_desc *descs_host, int n, void **plan);
int morph_batch_plan_launch(void *plan, void *stream);
int morph_batch_plan_destroy(void *plan);

/*
 * The paper has no counterpart to this entry point; it serves callers that
 * may not allocate device memory at all -- code whose device memory is owned
 * by another allocator or memory pool, real-time loops where cudaMalloc's
 * implicit synchronisation is not allowed, or plug-in hosts that hand over
 * only pre-allocated image buffers.  It runs the same batched persistent
 * kernel as morph_batch, but its scratch (per-image records, tensor maps, the
 * tile counter) lives in a fixed array in the library's device memory image,
 * which every GPU that loads the library keeps until the process exits.  It
 * calls no cudaMalloc/cudaFree and no allocating routine.
 *
 * At most MORPH_NOALLOC_MAX_IMAGES images per call (MORPH_ERR_LIMIT beyond).
 * The first call on a device looks up the array's device address (the
 * set-up), so make that first call before any stream capture.  All calls
 * share the one array and its host-side staging copy: calls that overlap on
 * the GPU, or run concurrently from several host threads, race.  The counter
 * the kernel schedules tiles with is reset on every call.  Asynchronous on
 * `stream`; descs_host may be reused when the call returns.
 */
#define MORPH_NOALLOC_MAX_IMAGES 256
int morph_batch_noalloc(const morph_desc *descs_host, int n, void *stream);

/*
 * Transpose (section 4): dst[x][y] = src[y][x].  src is width x height pixels
 * with src_pitch bytes per row; dst is height x width pixels (height pixels
 * per row, dst_pitch >= height * element size).  Device pointers, async.
 */
int transpose_u8(const uint8_t *src, int width, int height, size_t src_pitch,
                 uint8_t *dst, size_t dst_pitch, void *stream);
int transpose_u16(const uint16_t *src, int width, int height, size_t src_pitch,
                  uint16_t *dst, size_t dst_pitch, void *stream);

/*
 * Autotuner (section 5.3's crossover, measured here rather than taken from the
 * paper's ARM figures): times the candidate methods and tile shapes on the
 * current device, stores the chosen crossover windows and tiles, and writes
 * them to cache_path as JSON when it is not NULL.  When cache_path names an
 * existing, valid cache for this device it is loaded instead of re-measured.
 * Without a call the library uses built-in defaults.  Synchronous.
 */
int morph_autotune(const char *cache_path);

/*
 * Manual tuning (what morph_autotune sets): for dtype (MORPH_U8/MORPH_U16),
 * the pass along x uses the direct method of section 5.2.2 iff wx <=
 * cross_row and van Herk/Gil-Werman otherwise; the pass along y likewise with
 * wy and cross_col (section 5.3's w_x^0 and w_y^0); a negative crossover
 * keeps the current value.  tile_cfg selects the output tile per CTA when it
 * fits the window in shared memory (0: 128x64, 1: 64x64, 2: 64x128,
 * 3: 256x32, 4: 32x32, 5: 128x128, 6: 256x64, 7: 32x128 pixels); -1 lets a
 * built-in cost model pick
 * per call.  The result never changes, only the speed.  morph_reset_tuning
 * restores the built-in defaults.
 */
int morph_set_tuning(int dtype, int cross_row, int cross_col, int tile_cfg);
int morph_reset_tuning(void);

/*
 * Form of single-image calls with a 2-D window (section 5: the element is
 * separable, so erosion by wx x wy is erosion by 1 x wy followed by wx x 1).
 * mode -1 (default): two launches through an intermediate image the
 * library allocates stream-ordered for images of at least 2 Mpixels when
 * both passes take the van Herk/Gil-Werman method (both window sides above
 * the crossovers of morph_set_tuning; there the single-pass kernels were
 * measured faster than the fused kernel on the GB300), or when the fused
 * tile is so large that fewer than 3 CTAs fit on an SM; otherwise both
 * passes fused in one kernel.  0: always fused; 1:
 * always two launches.  The result never
 * changes.
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

/* Text for a morph_status value (static storage). */
const char *morph_status_string(int status);

/*
 * Number of kernel launches the library has enqueued since it was loaded, on
 * every device and stream (a launch captured into a CUDA graph counts once,
 * when captured).  For accounting: a caller can read it before and after a
 * call to learn how many kernels the call launched.  Never fails.  The paper
 * has no counterpart.
 */
long long morph_launch_count(void);

/*
 * Reads and clears the device error word that kernels set when a bounded wait
 * gives up (0 = none; 1 = a wait for a TMA load gave up).  Synchronises the
 * device.
 */
int morph_device_error(void);

/*
 * Self-test of that failure detection: launches one warp that waits, with
 * the kernels' bounded wait (2 s of the GPU's global timer), on an mbarrier
 * phase that nothing completes.  The wait gives up, the warp records error 1
 * in the device error word and returns, and the context stays usable: once
 * the stream reaches it (about 2 s later) morph_device_error() returns 1.
 * No fault, trap or unbounded wait is involved.  Returns MORPH_OK when the
 * launch was queued, MORPH_ERR_CUDA otherwise.
 */
int morph_selftest_wait_timeout(void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MORPH_H */
