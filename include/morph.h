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
 * (section 5.3) measured on this GPU.  Small windows (both passes direct) and
 * small images run both passes fused in one kernel; a 1-D window above the
 * crossover runs on the single-pass kernel of its axis; a 2-D window whose
 * passes both take van Herk/Gil-Werman, on images of at least 2 Mpixels
 * (4 Mpixels when only one pass takes it), runs as two launches, the pass
 * along x into an intermediate image and the pass along y from it (see
 * morph_set_split).
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
 *    along x (see morph_set_xpass), which take their intermediate image
 *    per call from the stream-ordered allocator (cudaMallocFromPoolAsync
 *    and cudaFreeAsync on the call's stream, from a memory pool the
 *    library creates per device and that keeps freed memory for the next
 *    call, so a warm caller maps no new memory; calls on different streams
 *    never share a block; under stream capture the block is a node of the
 *    graph, allocated by cudaMallocAsync).  morph_release_staging gives the
 *    pool's unused memory back.  morph_batch_noalloc allocates nothing at
 *    all.
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
 * step's).  The gradient of windows up to 5 x 5 (on an image at least as
 * large as the window) runs as one kernel that keeps both steps in shared
 * memory and allocates nothing: each pixel is read once and written once
 * (morph_set_composite_kernel extends that form to every window up to
 * 9 x 9 and every kind).  Otherwise the call runs two ordinary calls
 * through one scratch image of width x height pixels (pitch rounded to 16
 * bytes) from the library's stream-ordered pool, allocated and freed on the
 * stream, so the intermediate stays in L2 where it fits; the gradient's
 * subtraction is then an elementwise pass after the dilation.  Either form
 * is safe to capture in a CUDA graph.  Errors as morph_apply;
 * MORPH_ERR_ARG for another kind, MORPH_ERR_NOMEM when the scratch cannot be
 * allocated.
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

/*
 * n contiguous copies between host and device memory in the order of
 * `stream`, one cudaMemcpyAsync each (direction from the pointers), issued in
 * one call so that a caller moving many small images (the serving loop's
 * micro-batches) pays one call instead of n.  No counterpart in the paper.
 * Every entry is checked first (MORPH_ERR_NULL for a null pointer with a
 * non-zero size, MORPH_ERR_ARG for n < 0); nothing is queued then.
 * MORPH_ERR_CUDA when a copy cannot be queued (the earlier ones are).
 */
typedef struct {
    void *dst;
    const void *src;
    uint64_t bytes;
} morph_copy_desc;
int morph_copy_batch(const morph_copy_desc *copies, int n, void *stream);
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
/*
 * Frees the host-copy staging buffers and pipelines above and gives the
 * unused memory of the library's stream-ordered scratch pools back to the
 * driver (blocks of calls still queued stay valid).  Later calls recreate
 * what they need.  Returns MORPH_OK.
 */
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
 * Runs all n images on `stream` in at most six launches: images whose
 * windows take the direct method (or too small for the single-pass kernels)
 * in one persistent launch of the fused kernel; the passes along x of 1-D
 * windows and of 2-D windows whose pass along x is above the crossover in
 * one batched launch of the pass-along-x kernel (the 2-D ones into
 * intermediate images; a direct pass along x of a 2-D window whose pass
 * along y is above the crossover runs instead in the fused launch, as a
 * 1-D pass into its intermediate); the passes along y of 1-D windows and of
 * those 2-D windows (direct-method ones included) in batched launches of
 * the pass-along-y kernel (one per tile-size class).  An image
 * whose pass above the crossover reads a source those kernels cannot load
 * fast (rows not aligned to 8 pixels, base and pitch, for the pass along x;
 * base or pitch not a multiple of 16 bytes for the pass along y) runs as
 * its single call instead, after the batched launches, as do images above
 * the size set by morph_set_batch_alone.  Each image gets exactly the bytes
 * of its single call.  The descriptor array is on the
 * host; the call copies it (and the derived records) to a stream-ordered
 * device block (from the library's stream-ordered pool on `stream`, which
 * also holds the intermediates) through the library's pinned staging buffers, so descs may
 * be reused as soon as the call returns.  Asynchronous.
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
 * records (and the intermediates) in device memory at fixed addresses, which
 * the plan owns, and captures the batch's launches in a CUDA graph;
 * plan_launch replays it on `stream` (one cudaGraphLaunch).  The image
 * buffers must stay alive and at the same addresses until plan_destroy.
 * Replays of one plan must not overlap on the GPU (they share the
 * intermediates and the tile counter).
 */
int morph_batch_plan_create(const morph_desc *descs_host, int n, void **plan);
int morph_batch_plan_launch(void *plan, void *stream);
int morph_batch_plan_destroy(void *plan);

/*
 * The paper has no counterpart to this entry point; it serves callers that
 * may not allocate device memory at all -- code whose device memory is owned
 * by another allocator or memory pool, real-time loops where cudaMalloc's
 * implicit synchronisation is not allowed, or plug-in hosts that hand over
 * only pre-allocated image buffers.  It runs every image in the batched
 * persistent fused kernel (morph_batch sends 2-D windows above the crossover
 * through an intermediate image instead, which would need image-sized
 * scratch); its scratch (per-image records, tensor maps, the tile counter)
 * lives in a fixed array in the library's device memory image, which every
 * GPU that loads the library keeps until the process exits.  It calls no
 * cudaMalloc/cudaFree and no allocating routine.
 *
 * At most MORPH_NOALLOC_MAX_IMAGES images per call (MORPH_ERR_LIMIT beyond).
 * The first call on a device looks up the array's device address and
 * page-locks the library's host-side staging copy of the records
 * (cudaHostRegister of memory the library already holds; the set-up), so make
 * that first call before any stream capture.  The records then reach the
 * device by an asynchronous copy on `stream` that reads the staging copy when
 * it runs; before rewriting the staging copy, a call waits until the
 * previous call's copy has run.  All calls share the one array and the one
 * staging copy: calls that overlap on the GPU, or run concurrently from
 * several host threads, race.  The counter the kernel schedules tiles with
 * is reset on every call.  descs_host may be reused when the call returns.
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
 * Switches that force a particular kernel, launch form or order (for tests,
 * profiling and measurement) are declared in morph_tuning.h; none of them
 * changes a result.
 */

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
