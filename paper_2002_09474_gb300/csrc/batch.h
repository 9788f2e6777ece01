// Host-side interfaces of the batched kernel (not part of the public ABI).
#pragma once

#include <vector>

#include "morph_internal.h"
#include "morph_tile.cuh"

namespace morph {

// One image of a batch as the kernel reads it from device memory.
struct BatchImage {
  ImgArgs a;
  Geom g;
  int esz, op;
  int tiles_x;  // tiles per row of this image
  int tile0;    // tiles of all earlier images
};

// Host-side layout of a batch: tile shape, shared memory, per-image records
// and their tensor maps (two per image: input, output).
struct BatchHost {
  int cfg = -1, smem = 0, ntiles = 0;
  std::vector<BatchImage> imgs;
  std::vector<CUtensorMap> maps;
  // launch configuration, resolved before any stream capture
  int grid = 0;
  int* err = nullptr;
};

struct BatchImageIn {
  FusedLaunch L;  // planned single-image launch (window clipped, methods chosen)
};

// Chooses the batch's tile shape and fills the records; -1 if no shape fits.
int batch_prepare(const BatchImageIn* in, int n, BatchHost* out);
// Resolves grid size, error word and kernel attributes (no stream work).
cudaError_t batch_configure(BatchHost* h);
// Enqueues the counter reset and the persistent kernel on `stream`.
cudaError_t batch_enqueue(const BatchHost& h, const BatchImage* d_imgs, const CUtensorMap* d_maps,
                          int* d_counter, cudaStream_t stream);
int batch_take_device_error();
// Enqueues the counter reset and the persistent kernel for records already in
// device memory (no host-side containers involved).
cudaError_t batch_enqueue_raw(int cfg, int smem, int grid, int* err, int nimg, int ntiles,
                              const BatchImage* d_imgs, const CUtensorMap* d_maps, int* d_counter,
                              cudaStream_t stream);

// Shared with the single-image launcher: kernel arguments and tensor maps of
// one image for tile shape TX x TY.
void fill_img_args(const FusedLaunch& L, const Geom& g, int TX, int TY, ImgArgs* a, CUtensorMap* tin,
                   CUtensorMap* tout);

}  // namespace morph
