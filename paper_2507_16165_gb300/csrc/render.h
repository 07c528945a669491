// Host-side launch interface of the render kernels.
#pragma once

#include <cuda_runtime.h>

#include "bh_types.cuh"

namespace bhk {

struct LaunchShape {
  int num_sms;        // streaming multiprocessors of the device
  int block;          // threads per block
  int blocks_per_sm;  // 0: the occupancy limit of each kernel
  // Surrogate only: side stream (high priority) and fork / join events that
  // run the FP64 band pass next to the surrogate pass; band_ev[0..1] time it.
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t* band_ev = nullptr;
  int band_warps = 4;  // FP64 band warps per SM
  int band_rows = 0;   // image rows the band list covers (band list threads) ...
  int band_row0 = 0;   // ... starting at this row (rows numbered over all cameras)
  int mixed_part = 0;  // MIXED: 0 = the whole render, 1 = band list and FP64 band
                       // pass only, 2 = coherent and long-ray passes only
};

// Launch the kernels of one render (MIXED: band list and FP64 band pass,
// with the coherent pass as its programmatic dependent running beside it;
// coherent pass; long-ray pass) on `stream`.  ev[0..3], when non-null,
// are recorded before the first kernel and after each pass.
cudaError_t launch_render(const Params& p, int mode, const LaunchShape& ls, cudaStream_t stream,
                          cudaEvent_t* ev);

// The surrogate pass's dynamic shared memory (its tensor-core tiles): set
// before its launches on a device.
cudaError_t surrogate_kernel_setup();

// Launch a surrogate render: band pre-pass, FP64 band pass on the side
// stream, the surrogate pass (which lists the rays it does not answer), the
// integrator's lock-step pass over that list and the long-ray pass.
// ev[0..3]: start, after the surrogate pass, after the integrator passes,
// end.
cudaError_t launch_surrogate(const Params& p, const LaunchShape& ls, cudaStream_t stream,
                             cudaEvent_t* ev);

// Fill the 512 checker-sky cell colours of a scene (16 x 32, row i = theta
// cell, column j = phi cell) on `stream`.
cudaError_t fill_sky_lut(unsigned long long seed, float4* out, cudaStream_t stream);

// Launch only the coherent pass (mode MODE_FP32 or MODE_FP64).  With
// p.budget >= p.max_steps no ray is moved to the long-ray list, so the pass
// finishes every ray itself and needs no spill or band storage.
cudaError_t launch_coherent_only(const Params& p, int mode, const LaunchShape& ls,
                                 cudaStream_t stream);

}  // namespace bhk
