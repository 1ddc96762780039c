// qed_internal.h -- host-side context of libqed and the internal entry points
// shared between its translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qed.h"
#include "qed_device.cuh"

struct qed_ctx {
  qed_config cfg;
  int device;
  int num_sms;
  // table grids (l = ln chi rows; y = ln delta; kappa)
  qed::Grid gl, gy, gk, glp, gkp;
  // FP64 master tables
  double *R64, *F64, *Y64, *P64, *Yp64;
  // FP32 copies (QED_FP32)
  float *R32, *F32, *Y32, *P32, *Yp32;
  // scan state for stable appends / compaction
  unsigned long long *tile_state;
  unsigned int *sync;  // [0] tile counter, [1] done counter, [2] epoch
  int64_t max_tiles;
  int64_t *snap;       // [4] counts snapshotted at the start of a fused step
  uint8_t *heavy_flags;  // [max_tiles * TILE] main-pass deferral flags
  int *heavy_list;       // [max_tiles * TILE] ordered deferred slots
  int64_t *heavy_n;      // length of heavy_list
  qed_counters *d_counters;
  // persistent-grid sizes per kernel
  int grid_lepton, grid_photon, grid_compact;
  int64_t launches;
  // measurement hooks (qed_profile_begin/end): 3 events per profiled step
  cudaEvent_t *prof_ev;
  int prof_max, prof_n;
};

namespace qed {
int build_tables(qed_ctx *c, cudaStream_t st);
constexpr int TILE = 256;  // particles per tile = threads per block in the step kernels
}  // namespace qed
