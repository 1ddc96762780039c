// qed_batched.cu -- batched independent runs under a captured CUDA graph, and
// the autotuner of the persistent launch size.
#include <chrono>
#include <cstdio>
#include <cstring>

#include "qed_internal.h"

namespace qed {

__global__ void k_step_advance(int64_t *d_step) { *d_step += 1; }

__global__ void k_step_set(int64_t *d_step, int64_t v) { *d_step = v; }

// Alive photons per tag (run index).
__global__ void k_tag_count(const uint8_t *alive, const uint32_t *tag, const int64_t *d_n,
                            int n_runs, int64_t *out) {
  extern __shared__ unsigned long long s_cnt[];
  for (int r = threadIdx.x; r < n_runs; r += blockDim.x) s_cnt[r] = 0ull;
  __syncthreads();
  const int64_t n = *d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (alive[i]) {
      uint32_t t = tag[i];
      if (t < (uint32_t)n_runs) atomicAdd(&s_cnt[t], 1ull);
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n_runs; r += blockDim.x)
    if (s_cnt[r]) atomicAdd(reinterpret_cast<unsigned long long *>(&out[r]), s_cnt[r]);
}

}  // namespace qed

using namespace qed;

static int cu(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return QED_OK;
  fprintf(stderr, "libqed: %s: %s\n", what, cudaGetErrorString(e));
  return QED_ERR_CUDA;
}

// One step of the batched sequence: fused step, then removal of the dead
// photons by hole filling (only the photons that died are replaced).
static int one_step(qed_ctx *c, const qed_species *e, const qed_species *p, const qed_species *g,
                    const qed_fields *f, int64_t step, cudaStream_t st) {
  int rc = qed_step_fused(c, e, p, g, f, step, (qed_stream_t)st);
  if (rc == QED_OK) rc = qed_compact_fill(c, g, (qed_stream_t)st);
  return rc;
}

static void make_key(const qed_species *e, const qed_species *p, const qed_species *g,
                     const qed_fields *f, int steps, unsigned long long key[24]) {
  memset(key, 0, sizeof(unsigned long long) * 24);
  const qed_species *sp[3] = {e, p, g};
  int k = 0;
  for (int i = 0; i < 3; ++i) {
    key[k++] = (unsigned long long)(uintptr_t)sp[i]->x;
    key[k++] = (unsigned long long)(uintptr_t)sp[i]->d_n;
    key[k++] = (unsigned long long)sp[i]->capacity;
    key[k++] = (unsigned long long)(uintptr_t)sp[i]->tag;
    key[k++] = (unsigned long long)(uintptr_t)sp[i]->ex;
  }
  key[k++] = (unsigned long long)f->mode;
  key[k++] = (unsigned long long)(uintptr_t)f->grid;
  key[k++] = (unsigned long long)steps;
  unsigned long long eb[6];
  memcpy(eb, f->e, sizeof(double) * 3);
  memcpy(eb + 3, f->b, sizeof(double) * 3);
  for (int i = 0; i < 6 && k < 24; ++i) key[k++] = eb[i];
}

extern "C" int qed_run_batched(qed_ctx *c, const qed_species *e, const qed_species *p,
                               const qed_species *g, const qed_fields *f, int64_t step0,
                               int steps, int n_runs, int64_t *d_run_photons,
                               qed_stream_t stream) {
  if (!c || !e || !p || !g || !f || steps <= 0 || n_runs < 0 || n_runs > 12288 ||
      (d_run_photons && (!g->tag || n_runs == 0)))
    return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long key[24];
  make_key(e, p, g, f, steps, key);
  int rc = QED_OK;
  if (!c->graph_exec || memcmp(key, c->graph_key, sizeof(key)) != 0) {
    if (c->graph_exec) {
      cudaGraphExecDestroy(c->graph_exec);
      c->graph_exec = nullptr;
    }
    // capture on the context's own non-blocking stream (the caller's stream may
    // be the legacy default stream, which cannot be captured); the graph is
    // then launched on the caller's stream
    cudaStream_t cs = c->capture_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return cu(err, "qed_run_batched: begin capture");
    c->use_dstep = 1;
    for (int s = 0; s < steps && rc == QED_OK; ++s) {
      rc = one_step(c, e, p, g, f, 0, cs);
      if (rc == QED_OK) {
        k_step_advance<<<1, 1, 0, cs>>>(c->d_step);
        c->launches += 1;
      }
    }
    c->use_dstep = 0;
    err = cudaStreamEndCapture(cs, &graph);
    if (rc != QED_OK || err != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return rc != QED_OK ? rc : cu(err, "qed_run_batched: end capture");
    }
    err = cudaGraphInstantiate(&c->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
      c->graph_exec = nullptr;
      return cu(err, "qed_run_batched: instantiate");
    }
    memcpy(c->graph_key, key, sizeof(key));
  }
  k_step_set<<<1, 1, 0, st>>>(c->d_step, step0);
  cudaError_t err = cudaGraphLaunch(c->graph_exec, st);
  if (err != cudaSuccess) return cu(err, "qed_run_batched: launch");
  if (d_run_photons) {
    err = cudaMemsetAsync(d_run_photons, 0, sizeof(int64_t) * n_runs, st);
    if (err == cudaSuccess) {
      k_tag_count<<<c->num_sms * 2, 256, sizeof(unsigned long long) * n_runs, st>>>(
          g->alive, g->tag, g->d_n, n_runs, d_run_photons);
      err = cudaGetLastError();
    }
    if (err != cudaSuccess) return cu(err, "qed_run_batched: tag count");
  }
  return QED_OK;
}

// Mean milliseconds of `reps` steps (fused step + hole-filling compaction of
// the photons) after one untimed step at the current launch sizes.
static int time_steps(qed_ctx *c, const qed_species *e, const qed_species *p, const qed_species *g,
                      const qed_fields *f, int reps, int64_t &step, cudaEvent_t a, cudaEvent_t b,
                      cudaStream_t st, double *per) {
  int rc = one_step(c, e, p, g, f, step++, st);  // warm-up for this size
  if (rc != QED_OK) return rc;
  cudaEventRecord(a, st);
  for (int r = 0; r < reps && rc == QED_OK; ++r) rc = one_step(c, e, p, g, f, step++, st);
  cudaEventRecord(b, st);
  if (rc != QED_OK) return rc;
  float ms = 0.f;
  if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
    return QED_ERR_CUDA;
  *per = ms / reps;
  return QED_OK;
}

extern "C" int qed_autotune(qed_ctx *c, const qed_species *e, const qed_species *p,
                            const qed_species *g, const qed_fields *f, int reps, int *best_factor,
                            double *ms_out, qed_stream_t stream) {
  if (!c || !e || !p || !g || !f || reps <= 0 || !best_factor) return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return QED_ERR_CUDA;
  int saved[QED_TUNE_GROUPS];
  memcpy(saved, c->grid_factor, sizeof(saved));
  double best_ms = 1e300;
  int best = 0;
  int64_t step = 1000000;
  for (int factor = 1; factor <= 8; ++factor) {
    for (int k = 0; k < QED_TUNE_GROUPS; ++k) c->grid_factor[k] = factor;
    double per = 0.0;
    const int rc = time_steps(c, e, p, g, f, reps, step, a, b, st, &per);
    if (rc != QED_OK) {
      memcpy(c->grid_factor, saved, sizeof(saved));
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return rc;
    }
    if (ms_out) ms_out[factor - 1] = per;
    if (per < best_ms) {
      best_ms = per;
      best = factor;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  for (int k = 0; k < QED_TUNE_GROUPS; ++k) c->grid_factor[k] = best;
  *best_factor = best;
  return QED_OK;
}

extern "C" int qed_autotune_groups(qed_ctx *c, const qed_species *e, const qed_species *p,
                                   const qed_species *g, const qed_fields *f, int reps,
                                   qed_tuning *out, qed_stream_t stream) {
  if (!c || !e || !p || !g || !f || reps <= 0 || !out) return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return QED_ERR_CUDA;
  memset(out, 0, sizeof(*out));
  int saved[QED_TUNE_GROUPS], saved_sched[QED_SCHED_PARAMS];
  memcpy(saved, c->grid_factor, sizeof(saved));
  memcpy(saved_sched, c->sched, sizeof(saved_sched));
  int64_t step = 2000000;
  int rc = QED_OK;
  double best_ms = 1e300;
  // coordinate descent: one group at a time, the others at their current best
  for (int grp = 0; grp < QED_TUNE_GROUPS && rc == QED_OK; ++grp) {
    int best = 0;
    double best_g = 1e300;
    for (int factor = 1; factor <= QED_TUNE_MAX_FACTOR && rc == QED_OK; ++factor) {
      c->grid_factor[grp] = factor;
      double per = 0.0;
      rc = time_steps(c, e, p, g, f, reps, step, a, b, st, &per);
      if (rc != QED_OK) break;
      out->ms[grp][factor - 1] = per;
      if (per < best_g) { best_g = per; best = factor; }
    }
    c->grid_factor[grp] = best;
    best_ms = best_g;
  }
  // then the chain scheduling, one parameter at a time over fixed candidates
  // (the first of each list is its default)
  static const int cand[QED_SCHED_PARAMS][QED_SCHED_MAX_CANDIDATES] = {
      {16, 8, 12, 20, 24, 0}, {12, 4, 8, 16, 0, 0}, {8, 2, 4, 12, 0, 0},
      {8, 1, 4, 12, 16, 0},   {32, 16, 24, 33, 0, 0}};
  for (int k = 0; k < QED_SCHED_PARAMS && rc == QED_OK; ++k) {
    int best = cand[k][0];
    double best_k = 1e300;
    for (int j = 0; j < QED_SCHED_MAX_CANDIDATES && cand[k][j] && rc == QED_OK; ++j) {
      c->sched[k] = cand[k][j];
      double per = 0.0;
      rc = time_steps(c, e, p, g, f, reps, step, a, b, st, &per);
      if (rc != QED_OK) break;
      out->sched_tried[k][j] = cand[k][j];
      out->sched_ms[k][j] = per;
      if (per < best_k) { best_k = per; best = cand[k][j]; }
    }
    c->sched[k] = best;
    if (best_k < best_ms) best_ms = best_k;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != QED_OK) {
    memcpy(c->grid_factor, saved, sizeof(saved));
    memcpy(c->sched, saved_sched, sizeof(saved_sched));
    return rc;
  }
  memcpy(out->grid_factor, c->grid_factor, sizeof(out->grid_factor));
  memcpy(out->sched, c->sched, sizeof(out->sched));
  out->ms_per_step = best_ms;
  return QED_OK;
}

extern "C" int qed_set_tuning(qed_ctx *c, const qed_tuning *t) {
  if (!c || !t) return QED_ERR_ARG;
  for (int k = 0; k < QED_TUNE_GROUPS; ++k)
    if (t->grid_factor[k] < 0 || t->grid_factor[k] > 64) return QED_ERR_ARG;
  for (int k = 0; k < QED_SCHED_PARAMS; ++k)
    if (!sched_valid(k, t->sched[k])) return QED_ERR_ARG;
  memcpy(c->grid_factor, t->grid_factor, sizeof(c->grid_factor));
  memcpy(c->sched, t->sched, sizeof(c->sched));
  return QED_OK;
}
