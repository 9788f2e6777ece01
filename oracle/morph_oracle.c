/*
 * CPU oracle for grayscale erosion / dilation with a rectangular structuring
 * element -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the bench
 * may load this library.  The GPU library shares no code, header, table or
 * helper with it, and nothing here is ever called on the product path.
 *
 * What is computed (paper section 2, the erosion equation):
 *   erosion:  D(x,y) = min { S(x',y') : x' in [x-ax, x-ax+wx-1],
 *                                       y' in [y-ay, y-ay+wy-1],
 *                                       0 <= x' < W, 0 <= y' < H }
 *   dilation: the same with max (section 2, "similarly using maximum").
 * (ax, ay) is the anchor: the structuring element's cell that sits on the
 * output pixel, counted from the element's top-left corner.  The paper's
 * literal formula S(x - n + wx/2, ...), n in [0, wx-1], is the anchor
 * ax = ceil(wx/2) - 1; the library default is floor(wx/2); both agree for odd
 * windows.  Pixels outside the image are ignored (the paper only says edges
 * are "processed separately", section 5.1.2 / 5.2.2), which is the same as
 * padding with the operation's identity (max value for erosion, 0 for
 * dilation).
 *
 * Pixel types: 8-bit (esz = 1) as in the paper (section 5 intro), and 16-bit
 * (esz = 2) under the same definition.
 *
 * Functions:
 *   oracle_morph         -- the definition, brute force over the clipped
 *                           window (O(W*H*wx*wy)); the oracle proper.
 *   oracle_morph_points  -- the same definition at a list of sample points,
 *                           for images too large for the full brute force.
 *   oracle_sep_vhgw      -- independent checker: the separable form of
 *                           section 5 (a wx x 1 pass then a 1 x wy pass),
 *                           each pass by the van Herk / Gil-Werman recurrence
 *                           named in section 5.1.1 (block prefix g, block
 *                           suffix h, out = op(h[start], g[end])), with the
 *                           two extra image-size buffers section 5.1.1 notes.
 *   oracle_line_wedge    -- independent checker: 1-D sliding min/max over one
 *                           strided line with the monotone-deque ("wedge")
 *                           method, textbook, no relation to the above.
 *   oracle_transpose     -- D[j][i] = S[i][j] (section 4: matrix transpose).
 * Parity pins for all of them live in tests/ (golden hand-worked examples,
 * scipy.ndimage special cases, exhaustive binary images, invariants).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EARG (-1)

/* Read pixel (x, y) of an image with row pitch `pitch` bytes. */
static inline uint32_t px_get(const void *img, int esz, long long pitch, int x, int y)
{
    const unsigned char *row = (const unsigned char *)img + (long long)y * pitch;
    if (esz == 1)
        return row[x];
    return ((const uint16_t *)row)[x];
}

static inline void px_put(void *img, int esz, long long pitch, int x, int y, uint32_t v)
{
    unsigned char *row = (unsigned char *)img + (long long)y * pitch;
    if (esz == 1)
        row[x] = (unsigned char)v;
    else
        ((uint16_t *)row)[x] = (uint16_t)v;
}

/* Identity of the operation: the value that never changes a min (erosion)
 * or a max (dilation). */
static inline uint32_t identity_of(int op, int esz)
{
    uint32_t maxval = (esz == 1) ? 0xFFu : 0xFFFFu;
    return op == 0 ? maxval : 0u;
}

static inline uint32_t apply_op(int op, uint32_t a, uint32_t b)
{
    if (op == 0)
        return a < b ? a : b;
    return a > b ? a : b;
}

static int check_args(int esz, int W, int H, long long pitch, int wx, int wy,
                      int ax, int ay, int op)
{
    if (esz != 1 && esz != 2)
        return ORACLE_EARG;
    if (W < 1 || H < 1 || wx < 1 || wy < 1)
        return ORACLE_EARG;
    if (ax < 0 || ax >= wx || ay < 0 || ay >= wy)
        return ORACLE_EARG;
    if (pitch < (long long)W * esz)
        return ORACLE_EARG;
    if (op != 0 && op != 1)
        return ORACLE_EARG;
    return ORACLE_OK;
}

/* The erosion/dilation value at one output pixel, straight from the
 * definition: scan the structuring element placed with its anchor on (x, y)
 * and skip every cell that falls outside the image. */
static uint32_t morph_at(const void *src, int esz, int W, int H, long long pitch,
                         int wx, int wy, int ax, int ay, int op, int x, int y)
{
    uint32_t acc = identity_of(op, esz);
    for (int m = 0; m < wy; ++m) {
        int ys = y - ay + m;
        if (ys < 0 || ys >= H)
            continue;
        for (int n = 0; n < wx; ++n) {
            int xs = x - ax + n;
            if (xs < 0 || xs >= W)
                continue;
            acc = apply_op(op, acc, px_get(src, esz, pitch, xs, ys));
        }
    }
    return acc;
}

int oracle_morph(const void *src, int esz, int W, int H, long long pitch,
                 int wx, int wy, int ax, int ay, int op,
                 void *dst, long long dpitch)
{
    if (!src || !dst)
        return ORACLE_EARG;
    if (check_args(esz, W, H, pitch, wx, wy, ax, ay, op) != ORACLE_OK)
        return ORACLE_EARG;
    if (dpitch < (long long)W * esz)
        return ORACLE_EARG;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            px_put(dst, esz, dpitch, x, y,
                   morph_at(src, esz, W, H, pitch, wx, wy, ax, ay, op, x, y));
    return ORACLE_OK;
}

/* The definition evaluated at n sample points (xs[i], ys[i]); out[i] holds
 * the value widened to 32 bits. */
int oracle_morph_points(const void *src, int esz, int W, int H, long long pitch,
                        int wx, int wy, int ax, int ay, int op,
                        const int32_t *xs, const int32_t *ys, long long n,
                        uint32_t *out)
{
    if (!src || (n > 0 && (!xs || !ys || !out)))
        return ORACLE_EARG;
    if (check_args(esz, W, H, pitch, wx, wy, ax, ay, op) != ORACLE_OK)
        return ORACLE_EARG;
    for (long long i = 0; i < n; ++i)
        if (xs[i] < 0 || xs[i] >= W || ys[i] < 0 || ys[i] >= H)
            return ORACLE_EARG;
#pragma omp parallel for schedule(dynamic, 16)
    for (long long i = 0; i < n; ++i)
        out[i] = morph_at(src, esz, W, H, pitch, wx, wy, ax, ay, op, xs[i], ys[i]);
    return ORACLE_OK;
}

/* ---------------------------------------------------------------------------
 * Separable van Herk / Gil-Werman checker (section 5: a pass of a wx x 1
 * element, a pass of a 1 x wy element; section 5.1.1: each pass finds the
 * min/max over ranges of constant length w with the vHGW recurrence).
 *
 * One line of n samples (stride `stride` values in a uint32 work array) is
 * padded with the identity so that every window is complete:
 *   P[i] = line[i - a]  for a <= i < a + n, identity elsewhere, i in [0, n+w-1)
 *   out[x] = op(P[x], ..., P[x+w-1])
 * The padded line is cut into blocks of length w starting at 0.  Inside a
 * block g is the running op from the block's first sample (prefix) and h the
 * running op towards the block's last sample (suffix).  A window [x, x+w-1]
 * starts in one block and ends in the same or the next one, so
 *   out[x] = op(h[x], g[x+w-1]).
 * ------------------------------------------------------------------------- */
static void vhgw_line(const uint32_t *line, long long stride, int n, int w, int a,
                      int op, uint32_t ident, uint32_t *P, uint32_t *g, uint32_t *h,
                      uint32_t *out)
{
    int len = n + w - 1;
    for (int i = 0; i < len; ++i) {
        int j = i - a;
        P[i] = (j >= 0 && j < n) ? line[(long long)j * stride] : ident;
    }
    for (int start = 0; start < len; start += w) {
        int end = start + w < len ? start + w : len; /* one past the block */
        g[start] = P[start];
        for (int i = start + 1; i < end; ++i)
            g[i] = apply_op(op, g[i - 1], P[i]);
        h[end - 1] = P[end - 1];
        for (int i = end - 2; i >= start; --i)
            h[i] = apply_op(op, h[i + 1], P[i]);
    }
    for (int x = 0; x < n; ++x)
        out[x] = apply_op(op, h[x], g[x + w - 1]);
}

int oracle_sep_vhgw(const void *src, int esz, int W, int H, long long pitch,
                    int wx, int wy, int ax, int ay, int op,
                    void *dst, long long dpitch)
{
    if (!src || !dst)
        return ORACLE_EARG;
    if (check_args(esz, W, H, pitch, wx, wy, ax, ay, op) != ORACLE_OK)
        return ORACLE_EARG;
    if (dpitch < (long long)W * esz)
        return ORACLE_EARG;
    uint32_t ident = identity_of(op, esz);
    long long npx = (long long)W * H;
    /* Two image-size work buffers: the x-pass result and the y-pass result. */
    uint32_t *img = (uint32_t *)malloc(sizeof(uint32_t) * npx);
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * npx);
    int maxn = W > H ? W : H;
    int maxw = wx > wy ? wx : wy;
    int lenmax = maxn + maxw - 1;
    if (!img || !tmp) {
        free(img);
        free(tmp);
        return ORACLE_EARG;
    }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            img[(long long)y * W + x] = px_get(src, esz, pitch, x, y);
    int fail = 0;
#pragma omp parallel
    {
        uint32_t *P = (uint32_t *)malloc(sizeof(uint32_t) * lenmax);
        uint32_t *g = (uint32_t *)malloc(sizeof(uint32_t) * lenmax);
        uint32_t *h = (uint32_t *)malloc(sizeof(uint32_t) * lenmax);
        uint32_t *o = (uint32_t *)malloc(sizeof(uint32_t) * maxn);
        if (!P || !g || !h || !o) {
#pragma omp atomic write
            fail = 1;
        } else {
            /* pass along x (wx x 1 element): one line per row */
#pragma omp for
            for (int y = 0; y < H; ++y) {
                vhgw_line(img + (long long)y * W, 1, W, wx, ax, op, ident, P, g, h, o);
                for (int x = 0; x < W; ++x)
                    tmp[(long long)y * W + x] = o[x];
            }
            /* pass along y (1 x wy element): one line per column */
#pragma omp for
            for (int x = 0; x < W; ++x) {
                vhgw_line(tmp + x, W, H, wy, ay, op, ident, P, g, h, o);
                for (int y = 0; y < H; ++y)
                    img[(long long)y * W + x] = o[y];
            }
        }
        free(P);
        free(g);
        free(h);
        free(o);
    }
    if (!fail)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                px_put(dst, esz, dpitch, x, y, img[(long long)y * W + x]);
    free(img);
    free(tmp);
    return fail ? ORACLE_EARG : ORACLE_OK;
}

/* ---------------------------------------------------------------------------
 * 1-D sliding min/max with a monotone deque (textbook "wedge" method).
 * out[x] = op over line[j], j in [x-a, x-a+w-1] clipped to [0, n).
 * The deque holds indices whose values are strictly better (smaller for min,
 * larger for max) than every later index kept behind them.
 * ------------------------------------------------------------------------- */
int oracle_line_wedge(const uint32_t *line, long long stride, int n, int w, int a,
                      int op, uint32_t *out)
{
    if (!line || !out || n < 1 || w < 1 || a < 0 || a >= w || (op != 0 && op != 1))
        return ORACLE_EARG;
    int *dq = (int *)malloc(sizeof(int) * n);
    if (!dq)
        return ORACLE_EARG;
    int head = 0, tail = 0; /* live entries dq[head..tail) */
    int next = 0;           /* next index to push */
    for (int x = 0; x < n; ++x) {
        int lo = x - a, hi = x - a + w - 1;
        if (hi > n - 1)
            hi = n - 1;
        while (next <= hi) {
            uint32_t v = line[(long long)next * stride];
            while (tail > head) {
                uint32_t b = line[(long long)dq[tail - 1] * stride];
                int dominated = (op == 0) ? (b >= v) : (b <= v);
                if (!dominated)
                    break;
                --tail;
            }
            dq[tail++] = next++;
        }
        while (tail > head && dq[head] < lo)
            ++head;
        /* window [max(lo,0), hi] is never empty because 0 <= a < w */
        out[x] = line[(long long)dq[head] * stride];
    }
    free(dq);
    return ORACLE_OK;
}

/* Section 4: D[j][i] = S[i][j] for an H x W image (rows of W pixels). */
int oracle_transpose(const void *src, int esz, int W, int H, long long pitch,
                     void *dst, long long dpitch)
{
    if (!src || !dst || (esz != 1 && esz != 2) || W < 1 || H < 1)
        return ORACLE_EARG;
    if (pitch < (long long)W * esz || dpitch < (long long)H * esz)
        return ORACLE_EARG;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            px_put(dst, esz, dpitch, y, x, px_get(src, esz, pitch, x, y));
    return ORACLE_OK;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the OpenMP threads of later calls (n >= 1); for timing the oracle on
 * one core against all.  Returns the previous count. */
int oracle_set_threads(int n)
{
    const int prev = oracle_num_threads();
#ifdef _OPENMP
    if (n >= 1)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
    return prev;
}
