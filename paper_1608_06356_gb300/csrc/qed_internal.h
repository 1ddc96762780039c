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
  int64_t *pic_n;      // [2] lepton counts at the start of a qed_pic_step
  int64_t heavy_slots;   // block-tile slots of both lepton species
  uint8_t *heavy_flags;  // [heavy_slots] streaming-pass class flags
  int *heavy_list;       // [heavy_slots] ordered deferred slots
  int64_t *heavy_n;      // length of heavy_list (photon pass)
  // class list of the streaming lepton pass: per-chunk packed counts and
  // per-class offsets, class starts
  unsigned long long *cls_chunk_cnt;  // [cls_chunks]
  uint32_t *cls_chunk_off;            // [cls_chunks][5]
  int64_t *cls_off;                   // [8]
  int64_t cls_chunks;
  // sub-step passes: photons per entry, final gamma and emission records
  uint32_t *sub_cnt;  // [heavy_slots]
  void *sub_gf;       // Real [rec_cap]
  void *rec_e;        // Real [SUB_REC][rec_cap]
  uint32_t *rec_k;    // [SUB_REC][rec_cap]
  int64_t rec_cap;
  int64_t *sub_meta;  // [4] appends of the emission (or pair) entries, counts before them
  int64_t *fill_meta; // [2] count before and after a hole-filling compaction
  unsigned int *replay_n;  // entries the writing pass leaves to its replay launch
  unsigned long long *probe_state;  // [2] look-back words of qed_test_wait_expiry (tile 0 never published)
  // staging records of the flagged leptons (streaming pass -> later passes)
  void *stage;          // Stage<Real> [stage_cap] (64 B FP32, 128 B FP64)
  uint32_t *stage_tag;  // [stage_cap]
  int32_t *stage_idx;   // [heavy_slots]
  unsigned int *stage_n;
  int64_t stage_cap;
  qed_counters *d_counters;
  // persistent-grid sizes per kernel
  int grid_lepton, grid_photon, grid_compact;
  int64_t launches;
  // learned inverse CDF: FP32 weights, Adam moments, gradient, BF16 fragments,
  // per-CTA partial gradients and losses (one allocation)
  void *mlp_mem;
  float *mlp_w, *mlp_m, *mlp_v, *mlp_g, *mlp_partial;
  uint32_t *mlp_frag;
  float *mlp_fw;         // FP32 small layers in the inference layout (W1, b1, b2, b3, W4, b4)
  // learned-sampler emissions of the single-pass lepton step, deferred to a
  // dense pass: records (16 or 48 bytes), their count and the pass's CTA
  // counter
  float4 *net_rec;
  int64_t net_cap;  // float4 units
  unsigned long long *net_n;  // [0] records appended, [1] CTAs of the dense pass done
  double *mlp_loss;
  int mlp_parts, mlp_ready;
  int64_t mlp_step;
  // graph replay: device step counter read by the kernels when non-null
  int64_t *d_step;
  int use_dstep;
  cudaGraphExec_t graph_exec;
  cudaStream_t capture_stream;  // non-blocking stream the graph is captured on
  unsigned long long graph_key[24];
  // persistent-grid occupancy factor per kernel group (QED_TUNE_*; 0 = as
  // many CTAs per SM as fit)
  int grid_factor[QED_TUNE_GROUPS];
  // Method I chain scheduling (QED_SCHED_*; 0 = default)
  int sched[QED_SCHED_PARAMS];
  // host-resident lepton steps (qed_lepton_step_host): three staging buffers,
  // their device counts, pinned photon counts, input and output streams and
  // per-buffer events (copied in, stepped, copied out)
  void *hs_mem;
  size_t hs_per_buf;
  int64_t *hs_dn;
  int64_t *hs_cnt;
  cudaStream_t hs_in, hs_out;
  cudaEvent_t hs_ev[9];
  // bound of the photon emission rate used by the single-pass lepton kernel:
  // W_rad <= w_up_row[j] chi / gamma for ln chi >= row j of the rate table
  float *w_up_row;  // [gl.n] (device)
  // measurement hooks (qed_profile_begin/end): 3 events per profiled step
  cudaEvent_t *prof_ev;   // QED_PROF_MARKS events per profiled step
  int prof_max, prof_n;
  cudaEvent_t *prof_cur;  // the current fused step's events while it is launched, else null
};

namespace qed {
int build_tables(qed_ctx *c, cudaStream_t st);
int lepton_step_host(qed_ctx *c, const qed_species *lh, const qed_species *g,
                     const qed_species *gh, const qed_fields *f, int64_t step, int64_t chunk,
                     cudaStream_t st);
void free_host_step(qed_ctx *c);
int mlp_alloc(qed_ctx *c);
// CTAs per SM for a persistent launch of a kernel group: the occupancy limit,
// capped by the group's autotuned factor when one is set
inline int persistent_blocks_per_sm(const qed_ctx *c, int occupancy, int group) {
  int b = occupancy < 1 ? 1 : occupancy;
  const int f = c->grid_factor[group];
  if (f > 0 && f < b) b = f;
  return b;
}
// Defaults of the chain-scheduling parameters (QED_SCHED_*), and a
// parameter of the context or its default.
constexpr int SCHED_DEF_EMIT_LANES = 16, SCHED_DEF_ROUND_LANES = 12, SCHED_DEF_SCAN_DRAWS = 8,
              SCHED_DEF_SCAN_LEFT = 8, SCHED_DEF_QUEUE_TRIGGER = 32;
inline int sched_default(int k) {
  switch (k) {
    case QED_SCHED_EMIT_LANES: return SCHED_DEF_EMIT_LANES;
    case QED_SCHED_ROUND_LANES: return SCHED_DEF_ROUND_LANES;
    case QED_SCHED_SCAN_DRAWS: return SCHED_DEF_SCAN_DRAWS;
    case QED_SCHED_SCAN_LEFT: return SCHED_DEF_SCAN_LEFT;
    default: return SCHED_DEF_QUEUE_TRIGGER;
  }
}
inline int sched_param(const qed_ctx *c, int k) {
  const int v = c->sched[k];
  return v > 0 ? v : sched_default(k);
}
// Is v a valid value (0 = default) of scheduling parameter k?
inline bool sched_valid(int k, int v) {
  static const int hi[QED_SCHED_PARAMS] = {32, 32, 16, 32, 33};
  if (v == 0) return true;
  if (v < 1 || v > hi[k]) return false;
  return k != QED_SCHED_SCAN_DRAWS || (v >= 2 && v % 2 == 0);
}
// Event marks of a profiled fused step: 0 start, 1 after the lepton
// streaming pass, 2 after the class list, 3 after the counting pass, 4 after
// the scan, 5 after the writing pass (lepton stage done), 6 after the photon
// streaming pass, 7 after the photon stage.
constexpr int PROF_MARKS = QED_PROF_PHASES + 1;
inline cudaError_t prof_mark(qed_ctx *c, int k, cudaStream_t st) {
  return c->prof_cur ? cudaEventRecord(c->prof_cur[k], st) : cudaSuccess;
}
constexpr int TILE = 256;  // particles per tile = threads per block in the step kernels
constexpr int SUB_REC = 8; // emission records kept per particle by the sub-step counting pass
constexpr int CLS_CHUNK_FLAGS = 2048;  // flags per chunk of the class-list passes
}  // namespace qed
