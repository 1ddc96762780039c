// qed_api.cu -- the C ABI of libqed (declared in include/qed.h): argument
// checks, context life cycle, and the launch sequence of each call.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "qed_internal.h"

namespace qed {
template <class Real>
cudaError_t launch_lepton(qed_ctx *, const qed_species *, const qed_species *, const qed_species *,
                          const qed_fields *, int64_t, int, cudaStream_t);
template <class Real>
cudaError_t launch_photon(qed_ctx *, const qed_species *, const qed_species *, const qed_species *,
                          const int64_t *, const qed_fields *, int64_t, cudaStream_t);
template <class Real> cudaError_t launch_compact(qed_ctx *, const qed_species *, cudaStream_t);
template <class Real> cudaError_t launch_compact_fill(qed_ctx *, const qed_species *, cudaStream_t);
cudaError_t launch_count_alive(qed_ctx *, const qed_species *, int64_t *, cudaStream_t);
template <class Real>
cudaError_t launch_eval(qed_ctx *, int, int, const double *, const double *, const uint32_t *,
                        double *, int64_t, cudaStream_t);
cudaError_t launch_snapshot(qed_ctx *, const int64_t *, int64_t *, cudaStream_t);
cudaError_t launch_sample_xi(qed_ctx *, const float *, const float *, float *, int64_t, int64_t,
                             cudaStream_t);
cudaError_t launch_eval_xi_mlp(qed_ctx *, const double *, const double *, const uint32_t *, double *,
                               int64_t, cudaStream_t);
template <class Real>
cudaError_t launch_eval_chi(qed_ctx *, const qed_species *, double *, cudaStream_t);
cudaError_t launch_fill(qed_ctx *, float *, int, int, int, double, double, double, double,
                        cudaStream_t);
enum { MODE_PUSH_ = 0, MODE_EMIT_ = 1, MODE_FUSED_ = 2 };
}  // namespace qed

using namespace qed;

static int cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return QED_OK;
  fprintf(stderr, "libqed: %s: %s\n", what, cudaGetErrorString(e));
  return QED_ERR_CUDA;
}

extern "C" void qed_config_default(qed_config *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->a_S = 412148.45;  // m_e c^2 / (hbar omega0) at lambda = 1 um
  c->alpha = 1.0 / 137.035999;
  c->dt = 0.01;
  c->wdt_max = 0.2;
  c->xi_min_energy = 2.0;
  c->pair_sign = 1;
  c->precision = QED_FP32;
  c->chi_min = 1e-5;
  c->chi_max = 1e3;
  c->chi_pair_min = 2e-2;
  c->chi_pair_max = 1e3;
  c->fwd_per_unit = 0.0;
  c->inv_per_unit = 0.0;
  c->seed = 0;
  c->spec_lo = 2.0;
  c->spec_hi = 1000.0;
  c->max_particles = (int64_t)1 << 24;
  c->max_substeps = (int64_t)1 << 16;
}

extern "C" const char *qed_strerror(int code) {
  switch (code) {
    case QED_OK: return "ok";
    case QED_ERR_ARG: return "invalid argument";
    case QED_ERR_CUDA: return "CUDA runtime error";
    case QED_ERR_CAPACITY: return "size exceeds the context's capacity";
    case QED_ERR_DOMAIN: return "invalid table range";
    case QED_ERR_TIMEOUT: return "bounded device wait ran out";
    case QED_ERR_NOCONV: return "table build did not converge";
    case QED_ERR_NOMEM: return "device allocation failed";
    case QED_ERR_UNSUPPORTED: return "unsupported in this configuration";
    default: return "unknown error";
  }
}

static void free_ctx(qed_ctx *c) {
  if (!c) return;
  free_host_step(c);
  void *ptrs[] = {c->R64, c->F64, c->Y64, c->P64, c->Yp64, c->R32, c->F32, c->Y32,
                  c->P32, c->Yp32, c->tile_state, c->sync, c->snap, c->pic_n, c->d_counters,
                  c->heavy_flags, c->heavy_list, c->heavy_n, c->cls_chunk_cnt,
                  c->cls_chunk_off, c->cls_off, c->sub_cnt, c->sub_gf, c->rec_e,
                  c->rec_k, c->sub_meta, c->fill_meta, c->replay_n, c->stage, c->stage_tag,
                  c->stage_idx, c->stage_n, c->probe_state,
                  c->mlp_mem, c->w_up_row, c->net_rec, c->net_n};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  free(c);
}

static void prof_release(qed_ctx *c) {
  if (!c->prof_ev) return;
  for (int i = 0; i < PROF_MARKS * c->prof_max; ++i) cudaEventDestroy(c->prof_ev[i]);
  free(c->prof_ev);
  c->prof_ev = nullptr;
  c->prof_max = c->prof_n = 0;
}

extern "C" void qed_destroy(qed_ctx *c) {
  if (!c) return;
  cudaDeviceSynchronize();
  prof_release(c);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  if (c->d_step) cudaFree(c->d_step);
  free_ctx(c);
}

extern "C" int qed_profile_begin(qed_ctx *c, int max_steps) {
  if (!c || max_steps <= 0 || max_steps > 100000) return QED_ERR_ARG;
  prof_release(c);
  c->prof_ev = (cudaEvent_t *)calloc((size_t)PROF_MARKS * max_steps, sizeof(cudaEvent_t));
  if (!c->prof_ev) return QED_ERR_NOMEM;
  for (int i = 0; i < PROF_MARKS * max_steps; ++i) {
    cudaError_t e = cudaEventCreate(&c->prof_ev[i]);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(c->prof_ev[j]);
      free(c->prof_ev);
      c->prof_ev = nullptr;
      c->prof_max = c->prof_n = 0;
      return cuda_fail(e, "qed_profile_begin");
    }
  }
  c->prof_max = max_steps;
  c->prof_n = 0;
  return QED_OK;
}

extern "C" int qed_profile_end_phases(qed_ctx *c, double *ms, int64_t *steps) {
  if (!c || !c->prof_ev || !ms) return QED_ERR_ARG;
  for (int q = 0; q < QED_PROF_PHASES; ++q) ms[q] = 0.0;
  for (int k = 0; k < c->prof_n; ++k) {
    cudaEvent_t *ev = c->prof_ev + PROF_MARKS * k;
    cudaError_t e = cudaEventSynchronize(ev[QED_PROF_PHASES]);
    for (int q = 0; q < QED_PROF_PHASES && e == cudaSuccess; ++q) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
      ms[q] += t;
    }
    if (e != cudaSuccess) { prof_release(c); return cuda_fail(e, "qed_profile_end"); }
  }
  if (steps) *steps = c->prof_n;
  prof_release(c);
  return QED_OK;
}

extern "C" int qed_profile_end(qed_ctx *c, double *lepton_ms, double *photon_ms, int64_t *steps) {
  double ms[QED_PROF_PHASES];
  int rc = qed_profile_end_phases(c, ms, steps);
  if (rc != QED_OK) return rc;
  if (lepton_ms) *lepton_ms = ms[0] + ms[1] + ms[2] + ms[3] + ms[4];
  if (photon_ms) *photon_ms = ms[5] + ms[6];
  return QED_OK;
}

static bool cfg_valid(const qed_config *c) {
  return c && c->a_S > 0 && c->alpha > 0 && c->dt > 0 && c->wdt_max > 0 &&
         c->xi_min_energy >= 0 && (c->pair_sign == 1 || c->pair_sign == -1) &&
         (c->precision == QED_FP32 || c->precision == QED_FP64) && c->chi_min > 0 &&
         c->chi_max > c->chi_min && c->chi_pair_min > 0 && c->chi_pair_max > c->chi_pair_min &&
         c->spec_lo > 0 && c->spec_hi > c->spec_lo && c->max_particles > 0 &&
         c->max_particles <= ((int64_t)1 << 30) - 4096 && c->max_substeps >= 1 &&
         (c->sampler == QED_SAMPLER_TABLE ||
          (c->sampler == QED_SAMPLER_MLP && c->precision == QED_FP32)) &&
         (c->generator == QED_GEN_METHOD_I || c->generator == QED_GEN_METHOD_II ||
          c->generator == QED_GEN_METHOD_III) &&
         (c->model == QED_MODEL_FORMULA_I || c->model == QED_MODEL_CLASSIC) &&
         (c->append_order == QED_APPEND_ORDERED || c->append_order == QED_APPEND_ANY);
}

// The single-pass lepton kernel's rate bounds: W_rad = (alpha a_S / gamma)
// (int_0^1 dW/dxi - int_0^xi_min dW/dxi) <= (alpha a_S / gamma) G(chi) with
// G = e^R from the rate table.  Between and beyond the table's nodes ln G is
// interpolated or extended with slope <= 1 in ln chi, so G(chi) / chi for
// ln chi >= l_j never exceeds the largest node value of e^(R - l) at nodes
// m >= j (w_up_row[j]; below the table G / chi is the first node's value).
// A 1% margin covers the cubic interpolation between nodes and FP32 rounding.
static int rate_bound(qed_ctx *c) {
  const int n = c->gl.n;
  double *R = (double *)malloc(sizeof(double) * (size_t)n);
  float *row = (float *)malloc(sizeof(float) * (size_t)n);
  if (!R || !row) { free(R); free(row); return QED_ERR_NOMEM; }
  cudaError_t e = cudaMemcpy(R, c->R64, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { free(R); free(row); return cuda_fail(e, "rate bound"); }
  const double k = 1.01 * c->cfg.alpha * c->cfg.a_S;
  double mx = 0.0;
  for (int j = n - 1; j >= 0; --j) {
    const double l = c->gl.x0 + j * c->gl.h;
    const double v = exp(R[j] - l);
    if (v > mx) mx = v;
    row[j] = (float)(k * mx);
  }
  free(R);
  if (cudaMalloc(&c->w_up_row, sizeof(float) * (size_t)n) != cudaSuccess) { free(row); return QED_ERR_NOMEM; }
  e = cudaMemcpy(c->w_up_row, row, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
  free(row);
  return cuda_fail(e, "rate bound");
}

extern "C" int qed_init_tables(const qed_config *cfg, qed_ctx **out, qed_stream_t stream) {
  if (!out || !cfg_valid(cfg)) return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  qed_ctx *c = (qed_ctx *)calloc(1, sizeof(qed_ctx));
  if (!c) return QED_ERR_NOMEM;
  c->cfg = *cfg;
  const bool f64 = cfg->precision == QED_FP64;
  // the classic spectrum's tail near xi = 1 varies like exp(-2 / (3 chi)) with
  // chi, so its FP32 rows need 2.5x the density for xi to 1e-5
  if (!(c->cfg.fwd_per_unit > 0))
    c->cfg.fwd_per_unit = f64 ? 16.0 : (cfg->model == QED_MODEL_CLASSIC ? 10.0 : 4.0);
  if (!(c->cfg.inv_per_unit > 0)) c->cfg.inv_per_unit = f64 ? 32.0 : 16.0;
  int rc = QED_OK;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) { free_ctx(c); return cuda_fail(e, "device query"); }

  // table grids, computed before allocation (identical to build_tables)
  {
    const double hf = 1.0 / c->cfg.fwd_per_unit, hk = 1.0 / c->cfg.inv_per_unit;
    auto mk = [](double lo, double hi, double h) {
      Grid g;
      int n_in = (int)ceil((hi - lo) / h - 1e-9);
      g.h = h; g.x0 = lo - 2.0 * h; g.n = n_in + 1 + 4; g.lo = lo; g.hi = lo + n_in * h;
      return g;
    };
    c->gl = mk(log(cfg->chi_min), log(cfg->chi_max), hf);
    // y = ln delta_min ~ ln(4 / (3 gamma chi)) falls with chi: the lower end
    // moves down with chi_max beyond 1e3 (gamma chi up to ~1e11 at chi = 1e5)
    const double y_lo = -18.0 - 1.5 * fmax(0.0, log(cfg->chi_max / 1e3));
    c->gy = mk(y_lo, 4.5, hf);
    c->gk = mk(-24.0, 4.75, hk);
    c->glp = mk(log(cfg->chi_pair_min), log(cfg->chi_pair_max), hf);
    c->gkp = mk(-23.0, 3.5, hk);
  }
  const size_t nR = c->gl.n, nF = (size_t)c->gl.n * c->gy.n, nY = (size_t)c->gl.n * c->gk.n,
               nP = c->glp.n, nYp = (size_t)c->glp.n * c->gkp.n;
  // FP32 forward + rate tables are staged in shared memory by the step kernels
  if (!f64 && 4 * (nR + nF) > 200 * 1024) { free_ctx(c); return QED_ERR_DOMAIN; }
  struct { void **p; size_t bytes; } allocs[] = {
      {(void **)&c->R64, nR * 8}, {(void **)&c->F64, nF * 8}, {(void **)&c->Y64, nY * 8},
      {(void **)&c->P64, nP * 8}, {(void **)&c->Yp64, nYp * 8},
      {(void **)&c->R32, f64 ? 0 : nR * 4}, {(void **)&c->F32, f64 ? 0 : nF * 4},
      {(void **)&c->Y32, f64 ? 0 : nY * 4}, {(void **)&c->P32, f64 ? 0 : nP * 4},
      {(void **)&c->Yp32, f64 ? 0 : nYp * 4}};
  for (auto &a : allocs) {
    if (!a.bytes) continue;
    if (cudaMalloc(a.p, a.bytes) != cudaSuccess) { free_ctx(c); return QED_ERR_NOMEM; }
  }
  // one look-back word per 32-particle warp tile of the sub-step pass (the
  // 256-particle block tiles of the other passes need fewer)
  c->max_tiles = (cfg->max_particles + 31) / 32 * 2 + 2;
  // the deferral flags and lists are indexed by 256-particle block-tile slots
  // of the two lepton species
  c->heavy_slots = ((cfg->max_particles + TILE - 1) / TILE * 2 + 2) * TILE;
  c->cls_chunks = c->heavy_slots / CLS_CHUNK_FLAGS + 1;
  // emission records for the first max_particles / 4 entries of the sub-step
  // list; later entries (and particles with more than SUB_REC photons) replay
  c->rec_cap = cfg->max_particles / 4 > 4096 ? cfg->max_particles / 4 : 4096;
  const size_t rsize = f64 ? sizeof(double) : sizeof(float);
  // staging records for the leptons the streaming pass defers (a record is
  // 16 words); past stage_cap a deferred particle is gathered from its arrays
  c->stage_cap = cfg->max_particles / 2 > 65536 ? cfg->max_particles / 2 : 65536;
  if (cudaMalloc(&c->tile_state, sizeof(unsigned long long) * c->max_tiles) != cudaSuccess ||
      cudaMalloc(&c->sync, sizeof(unsigned int) * 4) != cudaSuccess ||
      cudaMalloc(&c->snap, sizeof(int64_t) * 4) != cudaSuccess ||
      cudaMalloc(&c->pic_n, sizeof(int64_t) * 2) != cudaSuccess ||
      cudaMalloc(&c->d_counters, sizeof(qed_counters)) != cudaSuccess ||
      cudaMalloc(&c->heavy_flags, (size_t)c->heavy_slots + 4096) != cudaSuccess ||
      cudaMalloc(&c->heavy_list, sizeof(int) * (size_t)c->heavy_slots) != cudaSuccess ||
      cudaMalloc(&c->heavy_n, sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&c->cls_chunk_cnt, sizeof(unsigned long long) * (size_t)c->cls_chunks) != cudaSuccess ||
      cudaMalloc(&c->cls_chunk_off, sizeof(uint32_t) * 5 * (size_t)c->cls_chunks) != cudaSuccess ||
      cudaMalloc(&c->cls_off, sizeof(int64_t) * 8) != cudaSuccess ||
      cudaMalloc(&c->sub_cnt, sizeof(uint32_t) * (size_t)c->heavy_slots) != cudaSuccess ||
      cudaMalloc(&c->sub_gf, rsize * (size_t)c->rec_cap) != cudaSuccess ||
      cudaMalloc(&c->rec_e, rsize * SUB_REC * (size_t)c->rec_cap) != cudaSuccess ||
      cudaMalloc(&c->rec_k, sizeof(uint32_t) * SUB_REC * (size_t)c->rec_cap) != cudaSuccess ||
      cudaMalloc(&c->stage, 2 * 8 * rsize * (size_t)c->stage_cap) != cudaSuccess ||
      cudaMalloc(&c->stage_tag, sizeof(uint32_t) * (size_t)c->stage_cap) != cudaSuccess ||
      cudaMalloc(&c->stage_idx, sizeof(int32_t) * (size_t)c->heavy_slots) != cudaSuccess ||
      cudaMalloc(&c->stage_n, sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&c->sub_meta, 4 * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&c->fill_meta, 2 * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&c->replay_n, sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&c->probe_state, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    free_ctx(c);
    return QED_ERR_NOMEM;
  }
  e = cudaMemsetAsync(c->tile_state, 0, sizeof(unsigned long long) * c->max_tiles, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->sync, 0, sizeof(unsigned int) * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->snap, 0, sizeof(int64_t) * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, sizeof(qed_counters), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stage_n, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->probe_state, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) { free_ctx(c); return cuda_fail(e, "memset"); }
  // epoch starts at 1 so that zeroed state words never look valid
  unsigned int init_sync[4] = {0u, 0u, 1u, 0u};
  e = cudaMemcpyAsync(c->sync, init_sync, sizeof(init_sync), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { free_ctx(c); return cuda_fail(e, "init"); }
  if (cudaMalloc(&c->d_step, sizeof(int64_t)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    if (c->d_step) cudaFree(c->d_step);
    free_ctx(c);
    return QED_ERR_NOMEM;
  }
  rc = build_tables(c, st);
  if (rc == QED_OK) rc = rate_bound(c);
  if (rc == QED_OK) rc = mlp_alloc(c);
  if (rc != QED_OK) { free_ctx(c); return rc; }
  *out = c;
  return QED_OK;
}

static bool species_ok(const qed_species *s, bool need_alive) {
  if (!s) return false;
  if (s->capacity < 0) return false;
  if (s->capacity == 0) return s->d_n != nullptr;
  if (!s->x || !s->y || !s->z || !s->px || !s->py || !s->pz || !s->w || !s->id || !s->d_n)
    return false;
  if (need_alive && !s->alive) return false;
  return true;
}

static bool fields_ok(const qed_fields *f) {
  if (!f) return false;
  if (f->mode == QED_FIELDS_UNIFORM || f->mode == QED_FIELDS_PER_PARTICLE) return true;
  if (f->mode != QED_FIELDS_GRID) return false;
  return f->grid && f->nx > 0 && f->ny > 0 && f->nz > 0 && f->dx > 0 && f->dy > 0 && f->dz > 0 &&
         (((uintptr_t)f->grid) & 15) == 0;
}

static bool pp_fields_ok(const qed_species *s, const qed_fields *f) {
  if (f->mode != QED_FIELDS_PER_PARTICLE || s->capacity == 0) return true;
  return s->ex && s->ey && s->ez && s->bx && s->by && s->bz;
}

static int check_cap(const qed_ctx *c, const qed_species *s) {
  return s && s->capacity > c->cfg.max_particles ? QED_ERR_CAPACITY : QED_OK;
}

extern "C" int qed_gather_push(qed_ctx *c, const qed_species *s, const qed_fields *f, int64_t step,
                               qed_stream_t stream) {
  if (!c || !species_ok(s, false) || !fields_ok(f) || !pp_fields_ok(s, f) || s->q == 0)
    return QED_ERR_ARG;
  if (check_cap(c, s)) return QED_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = c->cfg.precision == QED_FP64
                      ? launch_lepton<double>(c, s, nullptr, s, f, step, MODE_PUSH_, st)
                      : launch_lepton<float>(c, s, nullptr, s, f, step, MODE_PUSH_, st);
  return cuda_fail(e, "qed_gather_push");
}

// Event generators II and III keep per-lepton state (od_p, od_r).
static bool od_ok(const qed_ctx *c, const qed_species *s) {
  return c->cfg.generator == QED_GEN_METHOD_I || !s || s->capacity == 0 || (s->od_p && s->od_r);
}

extern "C" int qed_emit(qed_ctx *c, const qed_species *l, const qed_species *g, const qed_fields *f,
                        int64_t step, qed_stream_t stream) {
  if (!c || !species_ok(l, false) || !species_ok(g, true) || !fields_ok(f) || !pp_fields_ok(l, f) ||
      l->q == 0 || !od_ok(c, l))
    return QED_ERR_ARG;
  if (check_cap(c, l) || check_cap(c, g)) return QED_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = c->cfg.precision == QED_FP64
                      ? launch_lepton<double>(c, l, nullptr, g, f, step, MODE_EMIT_, st)
                      : launch_lepton<float>(c, l, nullptr, g, f, step, MODE_EMIT_, st);
  return cuda_fail(e, "qed_emit");
}

extern "C" int qed_pair(qed_ctx *c, const qed_species *g, const qed_species *el,
                        const qed_species *po, const qed_fields *f, int64_t step,
                        qed_stream_t stream) {
  if (!c || !species_ok(g, true) || !species_ok(el, false) || !species_ok(po, false) ||
      !fields_ok(f) || !pp_fields_ok(g, f))
    return QED_ERR_ARG;
  if (check_cap(c, g) || check_cap(c, el) || check_cap(c, po)) return QED_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = c->cfg.precision == QED_FP64
                      ? launch_photon<double>(c, g, el, po, g->d_n, f, step, st)
                      : launch_photon<float>(c, g, el, po, g->d_n, f, step, st);
  return cuda_fail(e, "qed_pair");
}

extern "C" int qed_compact(qed_ctx *c, const qed_species *s, qed_stream_t stream) {
  if (!c || !species_ok(s, true)) return QED_ERR_ARG;
  if (check_cap(c, s)) return QED_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = c->cfg.precision == QED_FP64 ? launch_compact<double>(c, s, st)
                                                : launch_compact<float>(c, s, st);
  return cuda_fail(e, "qed_compact");
}

extern "C" int qed_compact_fill(qed_ctx *c, const qed_species *s, qed_stream_t stream) {
  if (!c || !species_ok(s, true)) return QED_ERR_ARG;
  if (check_cap(c, s)) return QED_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = c->cfg.precision == QED_FP64 ? launch_compact_fill<double>(c, s, st)
                                                : launch_compact_fill<float>(c, s, st);
  return cuda_fail(e, "qed_compact_fill");
}

extern "C" int qed_count_alive(qed_ctx *c, const qed_species *s, int64_t *d_count,
                               qed_stream_t stream) {
  if (!c || !d_count || !species_ok(s, true)) return QED_ERR_ARG;
  if ((((uintptr_t)d_count) & 7) != 0) return QED_ERR_ARG;
  return cuda_fail(launch_count_alive(c, s, d_count, (cudaStream_t)stream), "qed_count_alive");
}

extern "C" int qed_step_fused(qed_ctx *c, const qed_species *e, const qed_species *p,
                              const qed_species *g, const qed_fields *f, int64_t step,
                              qed_stream_t stream) {
  if (!c || !species_ok(e, false) || !species_ok(p, false) || !species_ok(g, true) ||
      !fields_ok(f) || !pp_fields_ok(e, f) || !pp_fields_ok(p, f) || !pp_fields_ok(g, f) ||
      !od_ok(c, e) || !od_ok(c, p))
    return QED_ERR_ARG;
  if (check_cap(c, e) || check_cap(c, p) || check_cap(c, g)) return QED_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  const bool f64 = c->cfg.precision == QED_FP64;
  const bool prof = c->prof_ev && c->prof_n < c->prof_max;
  c->prof_cur = prof ? c->prof_ev + PROF_MARKS * c->prof_n : nullptr;
  cudaError_t err = launch_snapshot(c, g->d_n, c->snap, st);
  if (err == cudaSuccess) err = prof_mark(c, 0, st);
  if (err == cudaSuccess)  // marks 1-5 inside
    err = f64 ? launch_lepton<double>(c, e, p, g, f, step, MODE_FUSED_, st)
              : launch_lepton<float>(c, e, p, g, f, step, MODE_FUSED_, st);
  if (err == cudaSuccess)  // mark 6 inside
    err = f64 ? launch_photon<double>(c, g, e, p, c->snap, f, step, st)
              : launch_photon<float>(c, g, e, p, c->snap, f, step, st);
  if (err == cudaSuccess) err = prof_mark(c, QED_PROF_PHASES, st);
  if (err == cudaSuccess && prof) c->prof_n += 1;
  c->prof_cur = nullptr;
  return cuda_fail(err, "qed_step_fused");
}

extern "C" int qed_lepton_step_host(qed_ctx *c, const qed_species *lh, const qed_species *g,
                                    const qed_species *gh, const qed_fields *f, int64_t step,
                                    int64_t chunk, qed_stream_t stream) {
  if (!c || !lh || !lh->d_n || !species_ok(g, true) || !fields_ok(f) || !pp_fields_ok(g, f) ||
      chunk <= 0)
    return QED_ERR_ARG;
  if (!lh->x || !lh->y || !lh->z || !lh->px || !lh->py || !lh->pz || !lh->w || !lh->id ||
      !pp_fields_ok(lh, f) || !od_ok(c, lh))
    return QED_ERR_ARG;
  if (f->mode == QED_FIELDS_PER_PARTICLE && !lh->ex) return QED_ERR_ARG;
  if (gh && (!gh->d_n || gh->capacity < g->capacity)) return QED_ERR_ARG;
  if (chunk > c->cfg.max_particles || check_cap(c, g)) return QED_ERR_CAPACITY;
  return lepton_step_host(c, lh, g, gh, f, step, chunk, (cudaStream_t)stream);
}

extern "C" int qed_sample_xi(qed_ctx *c, const float *chi, const float *gamma, float *xi, int64_t n,
                             int64_t step, qed_stream_t stream) {
  if (!c || n < 0 || (n > 0 && (!chi || !gamma || !xi))) return QED_ERR_ARG;
  if (c->cfg.precision != QED_FP32) return QED_ERR_UNSUPPORTED;
  if (n == 0) return QED_OK;
  return cuda_fail(launch_sample_xi(c, chi, gamma, xi, n, step, (cudaStream_t)stream),
                   "qed_sample_xi");
}

extern "C" int qed_rates(qed_ctx *c, int which, const double *chi, const double *gamma, double *W,
                         int64_t n, qed_stream_t stream) {
  if (!c || (which != 0 && which != 1) || n < 0 || (n > 0 && (!chi || !gamma || !W)))
    return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = c->cfg.precision == QED_FP64
                      ? launch_eval<double>(c, 0, which, chi, gamma, nullptr, W, n, st)
                      : launch_eval<float>(c, 0, which, chi, gamma, nullptr, W, n, st);
  return cuda_fail(e, "qed_rates");
}

extern "C" int qed_sample_table(qed_ctx *c, int which, const double *chi, const double *gamma,
                                const uint32_t *word, double *xi, int64_t n, qed_stream_t stream) {
  if (!c || which < 0 || which > 2 || n < 0 ||
      (n > 0 && (!chi || !word || !xi || (which != 1 && !gamma))))
    return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (which == 2) {  // the learned sampler (FP32 contexts with loaded weights)
    if (c->cfg.precision != QED_FP32) return QED_ERR_UNSUPPORTED;
    if (!c->mlp_ready) return QED_ERR_ARG;
    return cuda_fail(launch_eval_xi_mlp(c, chi, gamma, word, xi, n, st), "qed_sample_table");
  }
  cudaError_t e = c->cfg.precision == QED_FP64
                      ? launch_eval<double>(c, 1, which, chi, gamma, word, xi, n, st)
                      : launch_eval<float>(c, 1, which, chi, gamma, word, xi, n, st);
  return cuda_fail(e, "qed_sample_table");
}

extern "C" int qed_chi(qed_ctx *c, const qed_species *s, double *chi, qed_stream_t stream) {
  if (!c || !s || !chi || !s->d_n || !s->px || !s->py || !s->pz || !s->ex || !s->ey || !s->ez ||
      !s->bx || !s->by || !s->bz)
    return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = c->cfg.precision == QED_FP64 ? launch_eval_chi<double>(c, s, chi, st)
                                               : launch_eval_chi<float>(c, s, chi, st);
  return cuda_fail(e, "qed_chi");
}

extern "C" int qed_fill_standing_wave(qed_ctx *c, float *grid, int nx, int ny, int nz, double x0,
                                      double dx, double a0, double t, qed_stream_t stream) {
  if (!c || !grid || nx <= 0 || ny <= 0 || nz <= 0 || nx > 8192 || !(dx > 0) ||
      (((uintptr_t)grid) & 15) != 0)
    return QED_ERR_ARG;
  return cuda_fail(launch_fill(c, grid, nx, ny, nz, x0, dx, a0, t, (cudaStream_t)stream),
                   "qed_fill_standing_wave");
}

extern "C" int qed_table_get(qed_ctx *c, int which, double *host_out, size_t n, double *dims) {
  if (!c || which < 0 || which > 4) return QED_ERR_ARG;
  const Grid *ga = nullptr, *gb = nullptr;
  const double *src = nullptr;
  switch (which) {
    case 0: ga = &c->gl; src = c->R64; break;
    case 1: ga = &c->gl; gb = &c->gy; src = c->F64; break;
    case 2: ga = &c->gl; gb = &c->gk; src = c->Y64; break;
    case 3: ga = &c->glp; src = c->P64; break;
    case 4: ga = &c->glp; gb = &c->gkp; src = c->Yp64; break;
  }
  size_t total = (size_t)ga->n * (gb ? gb->n : 1);
  if (dims) {
    dims[0] = ga->n; dims[1] = gb ? gb->n : 1;
    dims[2] = ga->x0; dims[3] = ga->h;
    dims[4] = gb ? gb->x0 : 0.0; dims[5] = gb ? gb->h : 0.0;
  }
  if (n == 0) return QED_OK;
  if (!host_out || n < total) return QED_ERR_ARG;
  return cuda_fail(cudaMemcpy(host_out, src, total * sizeof(double), cudaMemcpyDeviceToHost),
                   "qed_table_get");
}

extern "C" int qed_read_counters(qed_ctx *c, qed_counters *out, qed_stream_t stream) {
  if (!c || !out) return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(out, c->d_counters, sizeof(qed_counters),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int rc = cuda_fail(e, "qed_read_counters");
  if (rc == QED_OK && (out->status & QED_STATUS_TIMEOUT)) return QED_ERR_TIMEOUT;
  return rc;
}

extern "C" int qed_reset_counters(qed_ctx *c, qed_stream_t stream) {
  if (!c) return QED_ERR_ARG;
  return cuda_fail(cudaMemsetAsync(c->d_counters, 0, sizeof(qed_counters), (cudaStream_t)stream),
                   "qed_reset_counters");
}

// One decoupled look-back (one warp) for tile 1 behind a tile 0 whose state
// word stays zero -- never published, so never valid for epoch 1: lane 0 polls
// it until the spin limit, records QED_STATUS_TIMEOUT and the walk ends.
__global__ void k_wait_expiry(unsigned long long *words, qed_counters *cnt) {
  const ScanState S{words, nullptr, 2};
  uint32_t status = 0;
  lookback_warp(S, 1, 1u, 0u, status);
  if (threadIdx.x == 0 && status) atomicOr(&cnt->status, status);
}

extern "C" int qed_test_wait_expiry(qed_ctx *c, qed_stream_t stream) {
  if (!c) return QED_ERR_ARG;
  k_wait_expiry<<<1, 32, 0, (cudaStream_t)stream>>>(c->probe_state, c->d_counters);
  c->launches += 1;
  return cuda_fail(cudaGetLastError(), "qed_test_wait_expiry");
}

extern "C" int qed_last_device_status(qed_ctx *c, uint32_t *bits, int64_t *dropped) {
  if (!c) return QED_ERR_ARG;
  qed_counters h;
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, c->d_counters, sizeof(qed_counters), cudaMemcpyDeviceToHost);
  int rc = cuda_fail(e, "qed_last_device_status");
  if (rc != QED_OK) return rc;
  if (bits) *bits = h.status;
  if (dropped) *dropped = h.dropped;
  return (h.status & QED_STATUS_TIMEOUT) ? QED_ERR_TIMEOUT : QED_OK;
}

extern "C" int64_t qed_launch_count(const qed_ctx *c) { return c ? c->launches : 0; }
