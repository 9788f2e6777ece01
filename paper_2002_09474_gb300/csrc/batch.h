// Host-side interfaces of the batched kernels (not part of the public ABI).
#pragma once

#include <cstddef>
#include <vector>

#include "../../include/morph.h"
#include "morph_colv.cuh"
#include "morph_internal.h"
#include "morph_rowv.cuh"
#include "morph_tile.cuh"

namespace morph {

// One image of the fused group as the fused batch kernel reads it.
struct BatchImage {
  ImgArgs a;
  Geom g;
  int esz, op;
  int tiles_x;  // tiles per row of this image
  int tile0;    // tiles of all earlier images
};

// One image (or the first pass of a 2-D image) of the pass-along-x group.
struct BatchRowv {
  RowvArgs a;
  int esz, op;
  int task0;  // warp tasks of all earlier records
};

// One image (or the second pass of a 2-D image) of the pass-along-y group.
struct BatchColv {
  ColvArgs a;
  int esz, op;
  int task0;  // warp tasks of all earlier records of its class
  int map;    // index of its input tensor map
};

// Tile classes of the pass-along-y group: a launch per class, its shared
// memory sized for the class's largest warp tile.
constexpr int kColvClasses = 4;
constexpr int kColvClassBoxes[kColvClasses] = {2, 4, 8, kCvMaxBox};
// Rows per warp of the pass-along-x group, and its resident warps per SM
// (4 warps a CTA, 8 CTAs an SM).
constexpr int kBatchRR = 2;
constexpr int kBatchRowvWps = 32;

// Host-side layout of a batch.  Images are split into three groups by the
// form a single call would take: windows whose passes take the direct method
// (and small images) run in the fused persistent kernel; a 2-D window whose
// pass along y takes van Herk/Gil-Werman runs as a pass along x into an
// intermediate image (on the pass-along-x kernel where that pass takes van
// Herk/Gil-Werman too, else as a 1-D record of the fused kernel) and a pass
// along y from it; 1-D windows run on the kernel of their pass.  One launch
// per group (per tile class for the pass along y), in the order fused, x, y.
struct BatchHost {
  // fused group
  int cfg = -1, smem = 0, ntiles = 0, grid = 0;
  std::vector<BatchImage> imgs;
  std::vector<CUtensorMap> maps;  // two per image: input, output
  int* err = nullptr;
  // pass-along-x group
  std::vector<BatchRowv> rows;
  int row_tasks = 0;
  // pass-along-y group, records sorted by class
  std::vector<BatchColv> cols;
  std::vector<CUtensorMap> col_maps;
  int col_first[kColvClasses] = {}, col_count[kColvClasses] = {}, col_tasks[kColvClasses] = {};
  // intermediate images of the 2-D images (bytes from the intermediate base)
  size_t inter_bytes = 0;
  struct Inter {
    int row, col;     // its pass-along-x record (-1: a fused record) and pass-along-y record
    int fused;        // the fused record of its pass along x (-1: a pass-along-x record)
    size_t off;       // bytes from the intermediate base
    long long pitch;  // bytes per row (16-byte multiple)
    int W, H, esz;
  };
  std::vector<Inter> inters;
  // the passes along x that run in the fused group into an intermediate
  // (their records are filled again once the intermediate is bound)
  std::vector<FusedLaunch> fused_x;  // parallel to the inters with fused >= 0, in order
};

// One descriptor, validated and planned as a single call would be.
struct BatchImageIn {
  FusedLaunch L;  // window clipped, methods chosen
};

// Validates and plans n descriptors into caller-supplied arrays: `out` (n
// entries) and `ranges` (2n entries of scratch for the overlap check).  No
// destination may overlap any other image's source or destination (images
// of one launch run concurrently).  Returns a morph_status.
struct BatchRange {
  uintptr_t lo, hi;
  int is_dst;
};
int plan_batch_into(const morph_desc* descs, int n, BatchImageIn* out, BatchRange* ranges);

// The fused group alone: chooses the tile shape shared by the n images and
// fills caller-supplied records (n) and tensor maps (2n); -1 if no shape
// fits every image.
int batch_prepare_fused(const FusedLaunch* const* Ls, int n, int* cfg, int* smem, int* ntiles, BatchImage* imgs,
                        CUtensorMap* maps);

// Sorts the images into the three groups and sizes the records and the
// intermediates (no device addresses needed yet); -1 on failure.
int batch_prepare(const BatchImageIn* in, int n, BatchHost* out);
// Fills the intermediate pointers (at `inter`, a device block of
// h->inter_bytes) into the records and encodes the tensor maps over them.
int batch_bind_intermediates(void* inter, BatchHost* h);
// Resolves grid sizes, error word and kernel attributes (no stream work).
cudaError_t batch_configure(BatchHost* h);

// Device layout of a batch's records in one block.
struct BatchDev {
  size_t maps_off, imgs_off, counter_off, rows_off, col_maps_off, cols_off, inter_off, bytes;
};
BatchDev batch_dev_layout(const BatchHost& h);
// Enqueues every launch of the batch, its records already at `base` in the
// layout above.
cudaError_t batch_enqueue(const BatchHost& h, uint8_t* base, const BatchDev& L, cudaStream_t stream);
int batch_take_device_error();
// Enqueues the counter reset and the fused persistent kernel for records
// already in device memory (no host-side containers involved).
cudaError_t batch_enqueue_raw(int cfg, int smem, int grid, int* err, int nimg, int ntiles,
                              const BatchImage* d_imgs, const CUtensorMap* d_maps, int* d_counter,
                              cudaStream_t stream);
// Grid of the fused persistent kernel for a tile shape and shared memory.
cudaError_t batch_fused_grid(int cfg, int smem, int ntiles, int* grid, int** err);

// Shared with the single-image launcher: kernel arguments and tensor maps of
// one image for tile shape TX x TY.
void fill_img_args(const FusedLaunch& L, const Geom& g, int TX, int TY, ImgArgs* a, CUtensorMap* tin,
                   CUtensorMap* tout);

// The arguments of one image's pass in the batched single-pass kernels;
// fill_gpu: shorter tasks, for a group too small to fill the GPU.
bool rowv_batch_args(const FusedLaunch& L, RowvArgs* a, bool fill_gpu = false);
bool colv_batch_args(const FusedLaunch& L, ColvArgs* a, CUtensorMap* map, bool fill_gpu = false);

// Whether a planned image runs as its own single call instead of in the
// batched launches: a pass by van Herk/Gil-Werman whose source the batched
// single-pass kernels cannot load fast (rows not aligned for the
// pass-along-x kernel's vector loads, or not describable by TMA for the
// pass along y).
bool batch_runs_alone(const FusedLaunch& L);

// Whether TMA can describe an image at src with rows of pitch bytes: base
// and pitch multiples of 16 bytes.
inline bool tma_loadable(const void* src, long long pitch) {
  return reinterpret_cast<uintptr_t>(src) % 16 == 0 && pitch % 16 == 0;
}

}  // namespace morph
