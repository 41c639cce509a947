// amr.h -- device descriptors and launchers of the AMR level operations.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace mhd {

// One box item between two patch arrays: prolongation (a = coarse, b = fine)
// or restriction (a = fine, b = coarse); box in coarse global cell index.
struct DBoxItem {
  int32_t a, b;
  int32_t lo[3], ext[3];
};

// One flux-register capture on a patch: kind 0 = axis-normal faces (5 FP64
// planes over the box), kind 1 = axis edges (1 plane); box in the patch's
// array index space; mode 0 set, 1 add.
struct DCapture {
  int32_t patch, kind, axis, mode;
  int32_t lo[3], ext[3];
  double* dst;
};

// One deposit into a coarse patch's correction planes: box in coarse global
// index (faces: face index = index of the upper cell; edges: storing cell).
struct DDeposit {
  int32_t coarse, kind, axis, mode;  // mode 0: refluxing (ratio 2), 1: same-level synchronisation
  int32_t lo[3], ext[3];
  int32_t flo[3], fext[3];  // fine register box (fine global index)
  const double* fine;       // fine register (5 planes for faces, 1 for edges)
  const double* creg;       // coarse register over the box
  double* corr;             // correction planes of the coarse patch (18 planes)
  unsigned int* flags;      // the coarse patch's element flags (bytes, 4-aligned)
  int32_t corr_idx, pad2;   // index of the coarse patch's DCorr
};

// Correction planes of one coarse patch and its element flags (bit 0: the
// cell has a corrected face; bit 1 + a: face a has a corrected edge).
struct DCorr {
  int32_t patch, pad;
  int64_t count;  // 18 * nelem
  double* base;
  unsigned char* flags;  // zero outside a call: each call resets what it set
};

// The elements a refluxing call flags, one entry per element: (index into
// the call's DCorr array) << 40 | element index.
struct RefluxList {
  unsigned long long* entries;
  unsigned long long* count;
  unsigned long long capacity;
};

// A block table of an item list on the device (see list_elem): the blocks'
// tasks, the items' first elements (nitems + 1 entries), and whether the
// blocks are packed (small items share blocks) or aligned to the items.
struct PackedTasks {
  const BlockTask* tasks;
  const int64_t* starts;
  int nblocks, nitems;
  int packed;
};

// Ghost fill, one launch over the copies, one warp per task: rows row0 ..
// row0 + ghost_rows(dtype) x (32 / W) - 1 (row = y + ext_y z) of copy `copy`
// from x offset x0 (W = min(ext_x, 32); x0 a multiple of 32); excl holds each
// copy's bottom-layer rectangles (DCopy.xr, nx).  Restriction: pass 0 packed
// over the items, pass 1 over (item, axis) top layers (item 3 i + a).
struct GhostTask {
  int32_t copy, row0, x0, pad;
};
int ghost_rows(int dtype);
cudaError_t ghost_fill2_launch(int dtype, const DPatch* patches, const DCopy* copies, const DExcl* excl,
                               const GhostTask* tasks, int ntasks, const KernelTimer* tm, cudaStream_t s);
cudaError_t prolong_launch(int dtype, const DPatch* coarse, const DPatch* fine, const DBoxItem* items,
                           const PackedTasks& p, const KernelTimer* tm, cudaStream_t s);
cudaError_t restrict_launch(int dtype, const DPatch* fine, const DPatch* coarse, const DBoxItem* items,
                            const PackedTasks& p0, const PackedTasks& p1, const KernelTimer* tm, cudaStream_t s);
cudaError_t capture_launch(int dtype, const DPatch* patches, const DCapture* caps, const PackedTasks& p,
                           const void* scratch, const double* d_dt, const KernelTimer* tm, cudaStream_t s);
// Refluxing: deposits (flagging the elements they affect into `list`), the
// correction of the listed elements (which also clears their flags), and the
// zeroing of the deposited plane elements.
cudaError_t reflux_launch(int dtype, const DPatch* coarse, const DCorr* corr, const RefluxList& list,
                          const DDeposit* deps, const BlockTask* dep_tasks, int ndep, const KernelTimer* tm,
                          cudaStream_t s);

}  // namespace mhd
