// regrid.h -- device records of the data transfer into a new iteration of a
// level (regrid.cu) and their launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace mhd {

// One copy from an old patch (src) to a new patch (dst): kind -1 the cells of
// the box, kind a the axis-a faces of the box (global indices of the level).
struct DTransfer {
  int32_t src, dst, kind, pad;
  int32_t lo[3], ext[3];
};

// One prolongation box (coarse global indices) from coarse patch `coarse`
// into new fine patch `fine`, under a mask of one byte per coarse cell of the
// box [mlo, mlo + mext).
struct DProlongNew {
  int32_t coarse, fine;
  int32_t lo[3], ext[3];
  int32_t mlo[3], mext[3];
  const uint8_t* mask;
};

cudaError_t transfer_copy_launch(int dtype, const DPatch* old, const DPatch* fresh, const DTransfer* items,
                                 const BlockTask* tasks, int nblocks, cudaStream_t s);
cudaError_t prolong_new_launch(int dtype, const DPatch* coarse, const DPatch* fine, const DProlongNew* items,
                               const BlockTask* tasks, int nblocks, int energy_mode, unsigned long long* nfall,
                               cudaStream_t s);

}  // namespace mhd
