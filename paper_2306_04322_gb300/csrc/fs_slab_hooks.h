// Internal hooks of fs_plan.cu that the slab decomposition (fs_slab.cu)
// builds on: a slab is two single plans, one over its rows and one over its
// kx columns.  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>

#include "fs.h"

namespace fs {

// Make the single plan p (over nx' = 2 cols x points and the global ny) the
// column plan of a slab whose columns start at global kx = kx_base of the
// global problem g.
cudaError_t slab_adopt_columns(fs_plan* p, int kx_base, const fs_params& g);
// One pass on p's stream: kind 0 row pass in `mode` (0 from spectra, 1 from
// real fields, 2 inverse only), kind 1 column pass.
cudaError_t slab_pass(fs_plan* p, int kind, int mode);
void* slab_spec(fs_plan* p);     // [nf + 1][slot] packed half spectra
void* slab_real(fs_plan* p);     // nf real fields
double* slab_csum(fs_plan* p);   // FP64 sum of c carried for the k = 0 mode (FP32)
fs_status slab_read_flag(fs_plan* p);  // synchronise, read and clear the sticky device status

}  // namespace fs
