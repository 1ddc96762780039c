/*
 * qed.h -- C ABI of libqed, a GB300 (sm_103a) implementation of the
 * per-macroparticle QED Monte Carlo step of Wang, Sheng, Gibbon & Li,
 * "Modeling of photon and pair production due to QED effects in
 * particle-in-cell simulation" (arXiv:1608.06356).
 *
 * Physics (paper equation numbers):
 *   chi_e  -- Eq. (2);  chi_ph -- Eq. (3)
 *   photon emission spectrum, formula I -- Eq. (1), adopted by the paper for
 *     the simulation (text after Fig. 1)
 *   pair (Breit-Wheeler) spectrum -- Eq. (6)
 *   event generator: Method I (text before Eq. 7): emit iff W*Dt > r1; photon
 *     energy fraction from the inverse CDF, Eq. (7), with the infrared cut
 *     xi_min * eps_e = 2 m c^2
 *   adjustable time step (paragraph after Fig. 4): if W*Dt > 0.2 the generator
 *     runs N sub-steps with W*Dt/N <= 0.2
 *
 * Units: time 1/omega0, length c/omega0, momentum m_e c, fields m_e c omega0/e,
 * energies m_e c^2.  a_S is the Schwinger field E_S in field units.
 *
 * Conventions for every call:
 *   - Returns QED_OK (0) or a negative QED_ERR_* code; qed_strerror() names it.
 *   - Particle and field pointers are CALLER-OWNED DEVICE memory.  The library
 *     owns only what qed_init_tables allocates (tables, scan state, counters)
 *     and frees it in qed_destroy.  No call other than qed_init_tables
 *     allocates device memory.
 *   - Work is enqueued asynchronously on the given stream (NULL = legacy
 *     default stream).  Particle counts live on the device (qed_species.d_n),
 *     so no call reads them on the host and launches never depend on them.
 *   - Errors found on the device (capacity overflow, chi outside the table
 *     range, non-finite values, a bounded wait that ran out) never trap: they
 *     set bits in a device status word, read with qed_read_counters().
 *   - Calls that share a qed_ctx must be issued to one stream, or ordered.
 */
#ifndef QED_H
#define QED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *qed_stream_t; /* a cudaStream_t */
typedef struct qed_ctx qed_ctx;

/* ---- status codes ---------------------------------------------------- */
enum {
  QED_OK = 0,
  QED_ERR_ARG = -1,      /* invalid argument (NULL pointer, bad size, bad mode) */
  QED_ERR_CUDA = -2,     /* a CUDA runtime call failed */
  QED_ERR_CAPACITY = -3, /* a size exceeds what the context was built for */
  QED_ERR_DOMAIN = -4,   /* table range invalid */
  QED_ERR_TIMEOUT = -5,  /* a bounded device wait ran out (see status bits) */
  QED_ERR_NOCONV = -6,   /* table build did not converge */
  QED_ERR_NOMEM = -7,    /* device allocation failed (qed_init_tables only) */
  QED_ERR_UNSUPPORTED = -8
};

/* ---- device status bits (qed_counters.status) ----------------------- */
enum {
  QED_STATUS_CAPACITY = 1u, /* appends beyond a species' capacity were dropped */
  QED_STATUS_DOMAIN = 2u,   /* chi (or delta_min) outside the table range: clamped */
  QED_STATUS_NONFINITE = 4u,/* non-finite momentum or field met (particle skipped) */
  QED_STATUS_TIMEOUT = 8u,  /* a look-back wait hit its iteration limit */
  QED_STATUS_SUBSTEPS = 16u,/* sub-step count was capped at qed_config.max_substeps */
  QED_STATUS_REPLAY = 32u   /* a replayed emission chain found fewer photons than its
                               counting pass (should not happen); the missing photons
                               were written with zero energy */
};

enum { QED_FP32 = 0, QED_FP64 = 1 };
enum { QED_SAMPLER_TABLE = 0, QED_SAMPLER_MLP = 1 };
/* photon event generators (text around Fig. 2): Method I (default; W Dt/N > r1
 * with sub-steps), Method II (cumulative probability P_cum += W Dt, emit when
 * 1 - exp(-P_cum) > r3), Method III (emit when P_cum > r3, as printed). */
enum { QED_GEN_METHOD_I = 0, QED_GEN_METHOD_II = 1, QED_GEN_METHOD_III = 2 };
/* photon spectrum the tables are built from: formula I (Eq. 1; formula II,
 * Eq. 4, is the same function) or the classic limit (Eq. 5) restricted to
 * photons below the lepton's energy (0 < xi < 1). */
enum { QED_MODEL_FORMULA_I = 0, QED_MODEL_CLASSIC = 1 };
enum { QED_FIELDS_UNIFORM = 0, QED_FIELDS_PER_PARTICLE = 1, QED_FIELDS_GRID = 2 };
/* Order of the photons a lepton step appends (the paper prescribes none).
 * ORDERED: in a deterministic order -- by a class of the particle's sub-step
 *   count, then particle index, then sub-step -- so reruns give the same
 *   arrays bit for bit.
 * ANY: the same photons (ids, energies, positions, weights, fields) in an
 *   order that depends on the scheduling of the GPU's warps; the lepton step
 *   then runs in a single pass (FP32 contexts with event generator Method I;
 *   other contexts append in the ORDERED way).  Capacity overflow drops
 *   whichever appends come last. */
enum { QED_APPEND_ORDERED = 0, QED_APPEND_ANY = 1 };

/* ---- configuration ---------------------------------------------------- */
typedef struct {
  double a_S;           /* E_S / (m_e c omega0 / e); 412148.45 at lambda = 1 um */
  double alpha;         /* fine-structure constant, 1/137.035999 ("~1/137", Eq. 1) */
  double dt;            /* PIC step Dt in 1/omega0 */
  double wdt_max;       /* sub-step threshold: W*Dt/N <= wdt_max (0.2, after Fig. 4) */
  double xi_min_energy; /* infrared cut xi_min * eps_e = xi_min_energy (2 m c^2, Eq. 7) */
  int pair_sign;        /* sign of int K_{1/3} in Eq. (6): +1 (standard, default) or -1 (as printed) */
  int precision;        /* QED_FP32 (FP32 state/tables, FP64 chi where it cancels) or QED_FP64 */
  double chi_min, chi_max;           /* photon-emission table range in chi_e */
  double chi_pair_min, chi_pair_max; /* pair table range in chi_ph; below chi_pair_min W_pair = 0 */
  double fwd_per_unit;  /* forward-table nodes per unit of ln chi and ln delta (0 = default) */
  double inv_per_unit;  /* inverse-table nodes per unit of kappa (0 = default) */
  uint64_t seed;        /* Philox4x32-10 key */
  double spec_lo, spec_hi; /* photon-energy histogram: 64 log bins over [spec_lo, spec_hi) m c^2 */
  int64_t max_particles;   /* largest per-species capacity any call will use (sizes scan
                              state and the sub-step scratch, about 80 (FP32) or 120
                              (FP64) bytes per particle); default 2^24, at most
                              2^30 - 4096 */
  int64_t max_substeps;    /* cap on N per particle per step (status bit when hit) */
  int sampler;             /* QED_SAMPLER_TABLE (default) or QED_SAMPLER_MLP (FP32 contexts) */
  int generator;           /* QED_GEN_METHOD_I (default), _II or _III: photon event generator;
                              II and III need od_p, od_r on every lepton species */
  int model;               /* QED_MODEL_FORMULA_I (default) or QED_MODEL_CLASSIC */
  int append_order;        /* QED_APPEND_ORDERED (default) or QED_APPEND_ANY, see below */
} qed_config;

/* Fill *cfg with the paper-derived defaults (FP32, dt = 0.01, seed 0). */
void qed_config_default(qed_config *cfg);

/* ---- particle species (structure of arrays) ----------------------------
 * Element type of x..w and ex..bz is float in QED_FP32 contexts and double in
 * QED_FP64 contexts.  id: 64-bit particle ids (key of the Philox stream).
 * alive: photons only (1 alive, 0 dead); may be NULL for leptons.
 * ex..bz: per-particle fields (QED_FIELDS_PER_PARTICLE); children inherit
 * their parent's fields; NULL otherwise.
 * d_n: device int64 holding the current count; appends beyond `capacity` are
 * dropped and counted.  q: -1 electron, +1 positron, 0 photon.
 * tag: optional user tag (e.g. the index of an independent run), copied to the
 * particles a particle creates and moved by compaction; NULL if unused.
 * od_p, od_r: the state of event generators II and III (leptons; element type
 * as x): the cumulative probability P_cum and its random number r3, 0 meaning
 * "not drawn yet" (new leptons start at 0, 0).  NULL under Method I.        */
typedef struct {
  void *x, *y, *z, *px, *py, *pz, *w;
  uint64_t *id;
  uint8_t *alive;
  void *ex, *ey, *ez, *bx, *by, *bz;
  int64_t *d_n;
  int64_t capacity;
  int q;
  int pad_;
  uint32_t *tag;
  void *od_p, *od_r;
} qed_species;

/* ---- fields -------------------------------------------------------------
 * UNIFORM: e[3], b[3] everywhere.  PER_PARTICLE: the species' ex..bz arrays.
 * GRID: CIC (trilinear) gather from a periodic collocated node grid
 * grid[nz][ny][nx][8] (float; Ex Ey Ez Bx By Bz, 2 pad floats; node (i,j,k)
 * at (x0 + i dx, y0 + j dy, z0 + k dz)).                                     */
typedef struct {
  int mode, nx, ny, nz;
  double e[3], b[3];
  const float *grid;
  double dx, dy, dz, x0, y0, z0;
} qed_fields;

/* ---- counters (device-resident, accumulated until reset) --------------- */
typedef struct {
  int64_t emit_events;  /* photons emitted (Method I events of leptons) */
  int64_t pair_events;  /* pairs created */
  int64_t substeps;     /* generator sub-steps executed (leptons + photons) */
  int64_t dropped;      /* appends lost to capacity */
  int64_t domain;       /* evaluations clamped to the table range */
  uint32_t status;      /* QED_STATUS_* bits */
  uint32_t pad_;
  int64_t hist[64];     /* emitted-photon energies, 64 log bins over [spec_lo, spec_hi) */
  int64_t deferred;     /* leptons the streaming pass left to the emission passes
                           (an event possible or N > 1) */
} qed_counters;

const char *qed_strerror(int code);

/* Build the rate and inverse-CDF tables (FP64 on the device by Bessel
 * quadrature of Eqs. (1) and (6); FP32 copies for QED_FP32) and allocate the
 * context.  Blocks until the tables are built.  *out is set only on success. */
int qed_init_tables(const qed_config *cfg, qed_ctx **out, qed_stream_t stream);

/* Free everything the context owns (after synchronising its device work). */
void qed_destroy(qed_ctx *ctx);

/* Field gather + Boris push for all leptons of s (q = -1 or +1; photons
 * are pushed by qed_pair).  Positions advance by v*dt with the new momentum. */
int qed_gather_push(qed_ctx *ctx, const qed_species *s, const qed_fields *f, int64_t step,
                    qed_stream_t stream);

/* Method I photon emission (Eqs. 1, 2, 7) for every lepton of `lepton`
 * with fields gathered at its current position: chi_e, W_rad, N sub-steps,
 * events, xi draw, recoil, stable append of photons to `photons`. */
int qed_emit(qed_ctx *ctx, const qed_species *lepton, const qed_species *photons,
             const qed_fields *f, int64_t step, qed_stream_t stream);

/* Ballistic push + Method I Breit-Wheeler pair creation (Eqs. 3, 6) for every
 * alive photon present when the call starts; pairs appended in photon order,
 * the photon is marked dead. */
int qed_pair(qed_ctx *ctx, const qed_species *photons, const qed_species *electrons,
             const qed_species *positrons, const qed_fields *f, int64_t step,
             qed_stream_t stream);

/* Stable in-place removal of dead particles (alive == 0).  If a look-back
 * wait runs out (QED_STATUS_TIMEOUT), the tile that gave up writes nothing
 * and the count is left unchanged when it is the last tile: the species is
 * then not compacted (particles may be duplicated or stale) and must not be
 * used as the result. */
int qed_compact(qed_ctx *ctx, const qed_species *s, qed_stream_t stream);

/* Removal of dead particles that moves only as many particles as died.  With
 * a live particles left, the k-th dead slot below a (in index order) receives
 * the k-th live particle at or above a; live particles below a keep their
 * slot.  The result is deterministic; the order of the moved particles is not
 * their old order.  *s->d_n becomes a.  Same arguments and errors as
 * qed_compact. */
int qed_compact_fill(qed_ctx *ctx, const qed_species *s, qed_stream_t stream);

/* Number of live particles (alive != 0) among the first *s->d_n, written to
 * *d_count (device int64, 8-byte aligned) on `stream` without a host
 * synchronisation -- for counting particles between compactions. */
int qed_count_alive(qed_ctx *ctx, const qed_species *s, int64_t *d_count, qed_stream_t stream);

/* One fused QED-PIC step: electrons then positrons (gather at the old
 * position, Boris push, emission with the same fields), then the photons that
 * existed when the step began (push, pair creation).  Particles created in
 * this step are first advanced in the next one.  Any of e, p may have
 * capacity 0; g is required when e or p has particles. */
int qed_step_fused(qed_ctx *ctx, const qed_species *e, const qed_species *p,
                   const qed_species *g, const qed_fields *f, int64_t step,
                   qed_stream_t stream);

/* The lepton stage of qed_step_fused (gather at the old position, Boris
 * push, emission with recoil, photons appended to g) for leptons held in
 * HOST memory, streamed through the GPU in chunks of `chunk` leptons: chunk
 * k is copied in, stepped and copied back while the next is copied in and
 * the previous copied out (the caller's stream steps, two streams of the
 * context copy; the host arrays should be page-locked for the copies to
 * overlap).  Particle ids key the random draws, so the leptons and the set
 * of photons are those of one qed_step_fused call on the whole species with
 * no photons present at the start.
 *   l_host  a lepton species whose arrays (x..pz, w, id, the per-particle
 *           fields with QED_FIELDS_PER_PARTICLE, od_p/od_r with Methods
 *           II/III, optional tag) are HOST pointers and whose d_n points to a
 *           HOST int64 count; positions, momenta (and od_p/od_r) are updated
 *           in place.
 *   g       the photon species on the device; this call's photons are
 *           appended to it, chunk by chunk (photons present in g are not
 *           stepped).
 *   g_host  NULL, or a host mirror of g (host pointers for every array g has,
 *           capacity >= g's, d_n a HOST int64): the photons appended by this
 *           call are copied to the same indices and its count set.  When the
 *           device can map every mirror array (page-locked memory from the
 *           CUDA runtime), a kernel on the output stream copies each chunk's
 *           photons through the mapped pointers and the host waits only at
 *           the end; otherwise the host reads each chunk's photon count and
 *           queues the copies while the next chunk runs.
 * The context keeps three device staging buffers of `chunk` leptons
 * (allocated at the first call, grown by a later call that needs more).
 * Synchronous: returns when the leptons and photons are on the host.  The
 * context's counters accumulate over the chunks as over one step.  Calls on
 * one context share its staging buffers and must not overlap (other threads
 * included).  chunk must be in (0, max_particles] (QED_ERR_CAPACITY
 * otherwise); the call is refused inside a stream capture
 * (QED_ERR_UNSUPPORTED). */
int qed_lepton_step_host(qed_ctx *ctx, const qed_species *l_host, const qed_species *g,
                         const qed_species *g_host, const qed_fields *f, int64_t step,
                         int64_t chunk, qed_stream_t stream);

/* Isolated photon-energy sampler: xi[i] from Eq. (7) at (chi[i], gamma[i]),
 * r2 from Philox(seed; id = i, step, sub 0, stream 0) word 1 (float arrays,
 * device memory, QED_FP32 contexts). */
int qed_sample_xi(qed_ctx *ctx, const float *chi, const float *gamma, float *xi, int64_t n,
                  int64_t step, qed_stream_t stream);

/* Rates from the tables, for parity checks.  which = 0: W_rad(chi, gamma)
 * (photon emission with the xi_min cut); which = 1: W_pair(chi, gamma_ph).
 * Device double arrays; evaluated in the context's precision. */
int qed_rates(qed_ctx *ctx, int which, const double *chi, const double *gamma, double *W,
              int64_t n, qed_stream_t stream);

/* Inverse CDF at given inputs, for parity checks and the spectral error of
 * the learned sampler (Eq. 7).  which = 0: photon xi at (chi, gamma) for the
 * uniform word w (u = (w + 1/2) 2^-32) from the inverse table; which = 1: pair
 * xi at chi (Eq. 6; gamma unused, may be NULL); which = 2: photon xi as the
 * learned sampler gives it -- the network where (ln chi, kappa) is in its
 * domain, else the table -- in a QED_FP32 context whose weights are loaded
 * (QED_ERR_ARG before qed_mlp_load, QED_ERR_UNSUPPORTED in QED_FP64).  Device
 * arrays (double chi, gamma, xi; uint32 words); evaluated in the context's
 * precision. */
int qed_sample_table(qed_ctx *ctx, int which, const double *chi, const double *gamma,
                     const uint32_t *word, double *xi, int64_t n, qed_stream_t stream);

/* chi of every particle of s from its momentum and per-particle fields, for
 * parity checks: Eq. (2) (chi_e) when s->q != 0, Eq. (3) (chi_ph) when
 * s->q == 0, by the functions the step kernels use, in the context's precision
 * (QED_FP32: FP32, with the vector sum redone in FP64 where it cancels by more
 * than 2^7).  Needs px, py, pz and ex..bz; the count is read from s->d_n on the
 * device.  chi: device double[count]. */
int qed_chi(qed_ctx *ctx, const qed_species *s, double *chi, qed_stream_t stream);

/* Analytic standing wave (two counter-propagating circularly polarised waves
 * of amplitude a0 each) sampled at the nodes of a grid as qed_fields.GRID. */
int qed_fill_standing_wave(qed_ctx *ctx, float *grid, int nx, int ny, int nz, double x0,
                           double dx, double a0, double t, qed_stream_t stream);

/* Copy the FP64 master table `which` to host memory.  which: 0 photon
 * ln-rate R(l), 1 photon forward kappa(l, y), 2 photon inverse ln delta(l,
 * kappa), 3 pair ln-rate P(l), 4 pair inverse eta(l, kappa).  dims[0..5] gets
 * (n0, n1, x0_0, h_0, x0_1, h_1) as doubles; n may be 0 to query dims only.
 * Synchronous. */
int qed_table_get(qed_ctx *ctx, int which, double *host_out, size_t n, double *dims);

/* Counters: copy to host (synchronises `stream`) / zero them (async). */
int qed_read_counters(qed_ctx *ctx, qed_counters *out, qed_stream_t stream);
int qed_reset_counters(qed_ctx *ctx, qed_stream_t stream);

/* Device status since the last qed_reset_counters: `bits` gets the OR of the
 * QED_STATUS_* bits the kernels set, `dropped` the appends not written because
 * a species was full (either pointer may be NULL).  Waits for all work on the
 * context's device (cudaDeviceSynchronize), so it needs no stream.  Returns
 * QED_ERR_TIMEOUT when QED_STATUS_TIMEOUT is set (the outputs are still
 * written), QED_ERR_CUDA on a CUDA error. */
int qed_last_device_status(qed_ctx *ctx, uint32_t *bits, int64_t *dropped);

/* Failure-detection check of the bounded waits: launches one decoupled
 * look-back (one warp) behind a tile that never publishes, on two scratch
 * words of the context -- no particle data is touched.  The wait gives up at
 * its iteration limit (about a second), sets QED_STATUS_TIMEOUT and the kernel
 * returns, leaving the context usable.  Asynchronous on `stream`; read the
 * result with qed_last_device_status or qed_read_counters (both then return
 * QED_ERR_TIMEOUT) and clear it with qed_reset_counters. */
int qed_test_wait_expiry(qed_ctx *ctx, qed_stream_t stream);

/* ---- learned inverse CDF (surrogate for the tabulated inverse of Eq. 7) --
 * A 2 -> 64 -> 64 -> 64 -> 1 SiLU network maps x0 = (ln chi + 1.1512925)/5.7564627,
 * x1 = (kappa + 3.25)/6.75 to z; ln delta = z + 3 kappa - 2 ln(1 + e^kappa), where
 * kappa = ln(-ln(1 - u)) and delta = 2 xi/(3 chi (1 - xi)).  Domain chi in
 * [1e-3, 1e2], kappa in [-10, 3.5]; outside it the table is used.  Inference
 * runs in BF16 on the tensor cores with FP32 accumulation; training in FP32.
 * Parameters: 8577 floats, W1[2][64], b1[64], W2[64][64], b2[64], W3[64][64],
 * b3[64], W4[64], b4 (row index = input unit).  With sampler = QED_SAMPLER_MLP
 * emissions of particles with one sub-step (N = 1) and qed_sample_xi draw xi
 * with the network.
 *
 * qed_mlp_load: copy host weights in (resets the optimiser state).
 * qed_mlp_get:  copy the FP32 weights out.
 * qed_mlp_train: n_samples samples drawn on the device over the domain, targets
 *   from the FP64 inverse table; Adam (beta 0.9/0.999) with cosine decay from
 *   lr to lr/100; mini-batch 128 x 2 per CTA, one CTA per SM.  *final_loss gets
 *   the mean squared error of z over the last 8 steps.  Synchronous.
 * qed_mlp_grad: gradient of mean((z - t)^2) at the current weights for a given
 *   batch (device x[n][2], t[n]) into device grad[8577]; *loss (host) optional. */
int qed_mlp_load(qed_ctx *ctx, const float *host_w, size_t n);
int qed_mlp_get(qed_ctx *ctx, float *host_w, size_t n);
int qed_mlp_train(qed_ctx *ctx, int64_t n_samples, float lr, uint64_t seed, double *final_loss,
                  qed_stream_t stream);
int qed_mlp_grad(qed_ctx *ctx, const float *x, const float *t, int64_t n, float *grad,
                 double *loss, qed_stream_t stream);

/* Batched independent runs (many ensembles of uneven size advanced together).
 * The runs are concatenated in e, p, g (per-particle fields carry each run's
 * fields; tag holds the run index, 0 .. n_runs-1).  Advances `steps` fused
 * steps (qed_step_fused, then qed_compact_fill of the photons) starting at
 * step index step0, as one CUDA graph: captured on the first call for a given
 * combination of species, fields and steps, cached in the context and
 * replayed by later calls.  The step index is read by the kernels from a
 * device counter the graph advances, so every replay draws fresh numbers.
 * d_run_photons (device int64[n_runs], optional) receives the number of alive
 * photons per run after the last step.  The first call for a combination
 * captures the graph on `stream` (so it must not itself be capturing). */
int qed_run_batched(qed_ctx *ctx, const qed_species *e, const qed_species *p,
                    const qed_species *g, const qed_fields *f, int64_t step0, int steps,
                    int n_runs, int64_t *d_run_photons, qed_stream_t stream);

/* Autotuner of the persistent launches with one factor for every kernel group:
 * times `reps` fused steps (plus qed_compact_fill of the photons) for each
 * persistent-grid occupancy factor 1..8 on the given species -- which it
 * advances, so pass a disposable copy -- keeps the fastest factor in the
 * context (for every group) for all later launches and returns it in
 * *best_factor; per-candidate milliseconds go to ms_out[0..7] if non-NULL
 * (host).  factor 0 = as many CTAs per SM as fit.  qed_autotune_groups tunes
 * the groups separately. */
int qed_autotune(qed_ctx *ctx, const qed_species *e, const qed_species *p, const qed_species *g,
                 const qed_fields *f, int reps, int *best_factor, double *ms_out,
                 qed_stream_t stream);

/* Launch tuning by kernel group.  Every step kernel is a persistent launch of
 * a fixed block size (256 threads; the single-pass lepton kernel 128) whose
 * grid is the number of SMs times a number of CTAs per SM; that number, up to
 * what fits, is chosen per group of kernels:
 *   QED_TUNE_STREAM   lepton streaming: k_lepton_stream, the single-pass
 *                     lepton kernel, the push-only pass
 *   QED_TUNE_CHAINS   the ordered path's Method I chains (counting, replay)
 *   QED_TUNE_ORDER    the ordered path's lists, scans and writing pass
 *   QED_TUNE_PHOTON   photon streaming and pair passes
 *   QED_TUNE_COMPACT  stable compaction, the isolated sampler and the
 *                     learned sampler's dense pass of the single-pass step */
enum { QED_TUNE_STREAM = 0, QED_TUNE_CHAINS = 1, QED_TUNE_ORDER = 2, QED_TUNE_PHOTON = 3,
       QED_TUNE_COMPACT = 4, QED_TUNE_GROUPS = 5, QED_TUNE_MAX_FACTOR = 8 };

/* Scheduling of the Method I chains of the deferred leptons, run a warp at a
 * time with lanes in states (idle, rate, scanning, event pending) and one
 * state per round (the single-pass kernel's heavy phase, and the ordered
 * counting pass).  0 = the default, in brackets:
 *   QED_SCHED_EMIT_LANES     an emission round waits for this many lanes with
 *                            an event, 1..32 [16] (both paths)
 *   QED_SCHED_ROUND_LANES    a rate or scanning round of the single pass runs
 *                            with at least this many lanes, 1..32 [12]
 *   QED_SCHED_SCAN_DRAWS     Method I sub-steps drawn per lane per scanning
 *                            round, 2..16, even [8] (both paths; the single
 *                            pass draws four at a time)
 *   QED_SCHED_SCAN_LEFT      a scanning round of the single pass ends when
 *                            fewer lanes are still drawing, 1..32 [8]
 *   QED_SCHED_QUEUE_TRIGGER  queued deferred leptons that start a heavy phase
 *                            of the single pass, 1..33 [32]
 * The results (particles, photons, counters) do not depend on them. */
enum { QED_SCHED_EMIT_LANES = 0, QED_SCHED_ROUND_LANES = 1, QED_SCHED_SCAN_DRAWS = 2,
       QED_SCHED_SCAN_LEFT = 3, QED_SCHED_QUEUE_TRIGGER = 4, QED_SCHED_PARAMS = 5,
       QED_SCHED_MAX_CANDIDATES = 6 };
typedef struct {
  int grid_factor[QED_TUNE_GROUPS]; /* CTAs per SM per group; 0 = as many as fit */
  int sched[QED_SCHED_PARAMS];      /* chain scheduling (QED_SCHED_*); 0 = default */
  double ms_per_step;               /* one fused step + qed_compact_fill of the photons,
                                       with the chosen values */
  double ms[QED_TUNE_GROUPS][QED_TUNE_MAX_FACTOR]; /* per group, per factor 1..8 (the
                                       other groups at their values then; a factor beyond
                                       what fits runs as what fits) */
  int sched_tried[QED_SCHED_PARAMS][QED_SCHED_MAX_CANDIDATES]; /* candidate values of each
                                       scheduling parameter, in the order tried (0 = none) */
  double sched_ms[QED_SCHED_PARAMS][QED_SCHED_MAX_CANDIDATES]; /* their times */
} qed_tuning;

/* Autotuner by kernel group and chain scheduling: for each group in turn (the
 * order above), times `reps` fused steps plus qed_compact_fill of the photons
 * for every factor that fits (1..8 CTAs per SM), keeping the best before
 * tuning the next group; then each scheduling parameter in turn over a fixed
 * list of candidates.  The species are advanced -- pass disposable copies.
 * The chosen values are kept in the context for all later launches and
 * written, with the timings, to *out (host).  Synchronous. */
int qed_autotune_groups(qed_ctx *ctx, const qed_species *e, const qed_species *p,
                        const qed_species *g, const qed_fields *f, int reps, qed_tuning *out,
                        qed_stream_t stream);

/* Apply stored values (grid_factor and sched of *t; the timing fields are
 * ignored).  QED_ERR_ARG, and nothing applied, if a value is out of range. */
int qed_set_tuning(qed_ctx *ctx, const qed_tuning *t);

/* Measurement hooks.  qed_profile_begin creates CUDA events (call it outside
 * any timed or captured region) so that each of the next max_steps calls of
 * qed_step_fused records events on its stream between its phases:
 *   0 lepton streaming pass      1 lepton class list (3 launches)
 *   2 lepton counting pass       3 scan of the photon counts
 *   4 lepton writing pass        5 photon streaming pass
 *   6 photon list + ordered pass
 * qed_profile_end synchronises, returns the summed milliseconds of the
 * lepton stage (phases 0-4) and of the photon stage (5-6) and the number of
 * steps recorded, and releases the events; qed_profile_end_phases does the
 * same with the summed milliseconds of each phase in ms[0..QED_PROF_PHASES-1]. */
enum { QED_PROF_PHASES = 7 };
int qed_profile_begin(qed_ctx *ctx, int max_steps);
int qed_profile_end(qed_ctx *ctx, double *lepton_ms, double *photon_ms, int64_t *steps);
int qed_profile_end_phases(qed_ctx *ctx, double *ms, int64_t *steps);

/* Allocation-free stable compaction (no counterpart in the paper; it is a
 * service for callers that cannot allocate device memory -- an application
 * that owns every allocation through its own pool, a sandbox that forbids
 * cudaMalloc, or code where an allocation would synchronise the device).
 * Same result as qed_compact, but needs no qed_ctx: its only scratch (the
 * scan's look-back state and two counters) lives in a file-scope static
 * device array of 512 KiB per device, held until the process exits.
 *   s         species to compact in place (alive required; element type given
 *             by precision, QED_FP32 -> float, QED_FP64 -> double; the six
 *             field arrays are moved when all six are non-NULL)
 *   d_status  optional caller-owned device uint32 OR-ed with QED_STATUS_* bits
 * Returns QED_ERR_CAPACITY if s->capacity exceeds 16,777,216 particles; a count
 * *s->d_n above s->capacity is clamped to the capacity on the device and
 * reported as QED_STATUS_CAPACITY in *d_status.  After QED_STATUS_TIMEOUT the
 * species is not compacted (as for qed_compact).  Calls no allocating routine.  Every call shares the static array: calls that
 * overlap on the GPU race, so issue them to one stream or order them.  The
 * first call on a device performs a one-time set-up (cudaGetSymbolAddress of
 * the array with that device current); make it before any stream capture. */
int qed_compact_noalloc(const qed_species *s, int precision, uint32_t *d_status,
                        qed_stream_t stream);

/* ---- self-consistent fields: the particle-in-cell loop around the step ----
 * The paper adds its QED module to a PIC code (introduction) whose field
 * solver and current deposition it does not describe.  These calls close the
 * PIC cycle around the step with the standard explicit scheme: Maxwell's
 * equations on Yee's
 * staggered grid (K. S. Yee, IEEE Trans. Antennas Propag. 14, 302 (1966)),
 * leapfrogged in the units above,
 *     dB/dt = -curl E,      dE/dt = curl B - J,
 * J in units of e n_c c (n_c = eps0 m omega0^2 / e^2), with the current
 * deposited by the linear (CIC) shape at each component's staggered position.
 * The grid is periodic, nx*ny*nz cells, node (i,j,k) at (x0 + i dx, y0 + j dy,
 * z0 + k dz); every array below is float [nz][ny][nx] (x fastest) holding:
 *   ex, jx at (i+1/2, j, k)       bx at (i, j+1/2, k+1/2)
 *   ey, jy at (i, j+1/2, k)       by at (i+1/2, j, k+1/2)
 *   ez, jz at (i, j, k+1/2)       bz at (i+1/2, j+1/2, k)
 * nodes: the node grid of qed_fields.GRID (float [nz][ny][nx][8]) that the
 * particle steps gather from: E and B at the nodes, each the mean of the
 * component's two (E) or four (B) nearest staggered values.
 * All pointers are caller-owned device memory, 16-byte aligned.            */
typedef struct {
  int nx, ny, nz, pad_;
  double dx, dy, dz, x0, y0, z0;
  float *ex, *ey, *ez, *bx, *by, *bz;
  float *jx, *jy, *jz;
  float *nodes;
} qed_yee;

/* Add the current of the first min(*d_count, count of s) particles of s
 * (d_count: device int64, or NULL for all) to jx, jy, jz: each particle is a
 * charge s->q * w * weight_unit moving with v = p/gamma, taken at
 * x - v dt/2 (the middle of the step when x has just been advanced by v dt),
 * spread with the CIC weights of the staggered J positions and divided by
 * the cell volume dx dy dz.  weight_unit: real particles per unit of w,
 * divided by n_c (c/omega0)^3.  Element type of s as for the step
 * (qed_config.precision); the additions are float atomics, so their order --
 * and the last bits of J -- vary from run to run.  QED_ERR_ARG for photons
 * (q = 0) or a bad grid. */
int qed_pic_deposit(qed_ctx *ctx, const qed_species *s, const qed_yee *y, double weight_unit,
                    const int64_t *d_count, qed_stream_t stream);

/* advance != 0: one leapfrog step of the fields over the context's dt,
 *     B <- B - (dt/2) curl E;   E <- E + dt (curl B - J);   B <- B - (dt/2) curl E,
 * taking E, B from time n to n+1 with J at n+1/2; J is zeroed for the next
 * deposit.  Then (advance = 0: only) the nodes are written from E and B.
 * QED_ERR_ARG if dt breaks the Courant limit dt < 1/sqrt(1/dx^2 + 1/dy^2 +
 * 1/dz^2) or a grid argument is bad. */
int qed_pic_fields(qed_ctx *ctx, const qed_yee *y, int advance, qed_stream_t stream);

/* One cycle of the loop: qed_step_fused(e, p, g) gathering from y->nodes
 * (field mode GRID), then the current of the leptons that existed when the
 * call began (leptons created by this step's pairs are deposited from the
 * next step on), then qed_pic_fields(advance = 1).  The nodes must hold the
 * fields of the current time (qed_pic_fields with advance = 0 once at the
 * start).  e, p and g as for qed_step_fused (e and p leptons, either may have
 * capacity 0). */
int qed_pic_step(qed_ctx *ctx, const qed_species *e, const qed_species *p, const qed_species *g,
                 const qed_yee *y, double weight_unit, int64_t step, qed_stream_t stream);

/* Number of kernel launches this context has issued (for accounting). */
int64_t qed_launch_count(const qed_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* QED_H */
