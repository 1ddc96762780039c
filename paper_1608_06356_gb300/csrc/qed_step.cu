// qed_step.cu -- the per-macroparticle QED Monte Carlo step on sm_103a.
//
// What is computed per particle:
//   leptons: field gather (uniform / per-particle / CIC) -> Boris push ->
//            chi_e (Eq. 2) -> W_rad from the tables (Eq. 1 with the xi_min
//            cut) -> N = max(1, ceil(W Dt / 0.2)) sub-steps -> Method I events
//            with Philox draws -> xi from Eq. (7) -> recoil; photons appended.
//   photons: ballistic push -> chi_ph (Eq. 3) -> W_pair (Eq. 6) -> Method I ->
//            pair split xi (Eq. 6) -> e-/e+ appended, photon marked dead.
// How the lepton step is laid out: a streaming pass reads every particle once
// (coalesced), pushes it and decides with a cheap upper bound of the rate
// whether it surely has N = 1 and no event; those (most) are finished there.
// The rest are staged as 64-byte records, ordered by a class list (binned by
// N so that lanes of a warp do similar work), and run through a counting
// pass, a scan and a writing pass that append their photons in list order.
// Photons: a streaming pass, then an ordered pass over the flagged ones.
// Appends keep a deterministic order (and sub-step order within a particle);
// ordered passes scan within the block and across tiles by a single-pass
// decoupled look-back, so slot = count at launch + global prefix.
// Particle state is structure-of-arrays; loads and stores of a tile are
// coalesced 4-byte (FP32) or 8-byte (FP64) accesses.
#include <cstdio>

#include "qed_internal.h"
#include "qed_kernels.cuh"
#include "qed_mlp.cuh"

namespace qed {


// ---------------------------------------------------------------------------
// Lepton kernel (electrons and positrons in one launch)
// ---------------------------------------------------------------------------
// Pushed state of a flagged lepton, written once by the streaming pass so the
// later passes read 64 (FP32) or 128 (FP64) contiguous bytes per particle
// instead of gathering a 4- or 8-byte word from each of 14 arrays.
template <class Real> struct alignas(16) Stage {
  Real p[3], e[3], b[3];
  uint32_t id_lo, id_hi;
  Real w;
  Real x[3];
  uint32_t slot;
};
static_assert(sizeof(Stage<float>) == 64, "FP32 staging record");
static_assert(sizeof(Stage<double>) == 128, "FP64 staging record");
constexpr uint32_t STAGE_BATCH = 256;  // records a warp reserves at a time

template <class Real> struct LeptonArgs {
  Sp<Real> sp[2];
  int nsp;
  Sp<Real> ph;
  Fld<Real> f;
  Consts C;
  Tables<Real> T;  // R, F staged to shared memory; Y read through L1/L2
  Out o;
  int64_t step;
  uint8_t *heavy_flags;     // [streaming-pass slot] class flag (0 = finished)
  const int *heavy_list;    // class list: staging record or -(slot + 1), class-major
  const int64_t *heavy_n;   // length of heavy_list
  const int64_t *d_step;    // if set, the step index is read here (graph replay)
  const int64_t *cls_off;   // class list: class c occupies [cls_off[c-1], cls_off[c])
  Stage<Real> *stage;       // pushed state of the flagged leptons (streaming pass)
  uint32_t *stage_tag;      // their tags (species with tags)
  int32_t *stage_idx;       // [slot] staging index of a flagged slot, -1 if not staged
  unsigned int *stage_n;    // staging allocation counter (reset by the class-list scan)
  int64_t stage_cap;
  uint32_t *sub_cnt;        // sub-step passes: photons per class-2..5 entry
  Real *sub_gf;             // final gamma per entry (entries < rec_cap)
  Real *rec_e;              // [REC][rec_cap] photon energies
  uint32_t *rec_k;          // [REC][rec_cap] their sub-step indices
  int64_t rec_cap;
  const int64_t *sub_meta;  // [0] photons of the sub-step entries, [1] photon count before them
  int32_t *replay_list;     // entries whose chains the replay launch redoes
  unsigned int *replay_n;   // their number (reset by the scan)
  const uint32_t *mlp_frag; // learned inverse CDF (used when use_mlp)
  const float *mlp_w;
  int use_mlp;
  int emit_lanes, scan_draws;  // chain scheduling (QED_SCHED_EMIT_LANES, _SCAN_DRAWS)
};


// ---------------------------------------------------------------------------
// Push-only pass (qed_gather_push): field gather, Boris push and position
// update of every lepton; no emission, so no ordering is needed.
// ---------------------------------------------------------------------------
template <class Real, int FM>
__global__ void __launch_bounds__(TILE) k_lepton_push(LeptonArgs<Real> A) {
  __shared__ long long s_meta[2];
  if (threadIdx.x == 0) {
    s_meta[0] = *(volatile int64_t *)A.sp[0].d_n;
    s_meta[1] = A.nsp > 1 ? *(volatile int64_t *)A.sp[1].d_n : 0;
  }
  __syncthreads();
  const int64_t n0 = s_meta[0], n1 = s_meta[1];
  const Real dt = sel<Real>(A.C.dt, A.C.f_dt);
  uint32_t status = 0;
  for (int64_t g = blockIdx.x * (int64_t)TILE + threadIdx.x; g < n0 + n1;
       g += (int64_t)gridDim.x * TILE) {
    const int si = g < n0 ? 0 : 1;
    const Sp<Real> &S = A.sp[si];
    const int64_t i = si ? g - n0 : g;
    Real x = S.x[i], y = S.y[i], z = S.z[i];
    Real px = S.px[i], py = S.py[i], pz = S.pz[i];
    Real E[3], B[3];
    get_fields<Real, FM>(S, A.f, i, x, y, z, E, B);
    const Real gm = boris(px, py, pz, E, B, S.q, dt);
    if (!(gm < (Real)1e30)) {  // non-finite state: left as it was
      status |= QED_STATUS_NONFINITE;
      continue;
    }
    const Real ig = r_div(dt, gm);
    S.x[i] = x + px * ig; S.y[i] = y + py * ig; S.z[i] = z + pz * ig;
    S.px[i] = px; S.py[i] = py; S.pz[i] = pz;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) status |= __shfl_xor_sync(0xFFFFFFFFu, status, o);
  if ((threadIdx.x & 31) == 0 && status) atomicOr(&A.o.cnt->status, status);
}

// ---------------------------------------------------------------------------
// Streaming pass over all leptons: gather, push, chi, rate and the first
// Method I draw, with no block-wide synchronisation.  A particle that needs
// one sub-step and draws no event is finished here (its new position and
// momentum are written); the rest are only flagged -- 1: one sub-step with an
// event, 2: more than one sub-step -- and are redone, from their unchanged
// stored state, by the ordered passes that append photons.
// ---------------------------------------------------------------------------

template <class Real, int FM, int MODE>
__global__ void __launch_bounds__(TILE, sizeof(Real) == 4 ? 3 : 2) k_lepton_stream(LeptonArgs<Real> A) {
  const int64_t step_ = A.d_step ? *A.d_step : A.step;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kSmem = sizeof(Real) == 4;
  constexpr int NV = stream_words<FM>();
  Real *sR = kSmem ? reinterpret_cast<Real *>(smem_raw) : const_cast<Real *>(A.T.R);
  Real *sF = kSmem ? sR + A.T.gl.n : const_cast<Real *>(A.T.F);
  // prefetch buffers after the tables: [2][NV][TILE] words, then [2][TILE] ids
  const size_t tab_bytes = kSmem ? (((size_t)A.T.gl.n * (1 + A.T.gy.n) * sizeof(Real) + 15) & ~(size_t)15) : 0;
  Real *pf = reinterpret_cast<Real *>(smem_raw + tab_bytes);
  uint64_t *pf_id = reinterpret_cast<uint64_t *>(pf + 2 * NV * TILE);
  __shared__ long long s_meta[4];
  __shared__ BlockTally bt;
  if (kSmem) {
    load_tables_smem(sR, A.T.R, A.T.gl.n);
    load_tables_smem(sF, A.T.F, A.T.gl.n * A.T.gy.n);
  }
  block_tally_init(&bt);
  if (threadIdx.x == 0) {
    s_meta[0] = *(volatile int64_t *)A.sp[0].d_n;
    s_meta[1] = A.nsp > 1 ? *(volatile int64_t *)A.sp[1].d_n : 0;
  }
  __syncthreads();
  const int64_t n0 = s_meta[0], n1 = s_meta[1];
  const int64_t T0 = (n0 + TILE - 1) / TILE, T1 = (n1 + TILE - 1) / TILE;
  const int64_t nslots = (T0 + T1) * TILE;
  const Real inv_aS = sel<Real>(A.C.inv_aS, A.C.f_inv_aS);
  const Real dt = sel<Real>(A.C.dt, A.C.f_dt), wdt_max = sel<Real>(A.C.wdt_max, A.C.f_wdt_max);
  const int lane = threadIdx.x & 31;
  const int t = threadIdx.x;
  // this warp's current batch of staging records (warp-uniform)
  uint32_t batch_base = 0, batch_used = STAGE_BATCH;
  Tally tl;
  tl.clear();
  // issue the copies of slot `sl`'s particle into buffer b
  auto prefetch = [&](int64_t sl, int b) {
    const int64_t tile = sl / TILE;
    const int si = tile < T0 ? 0 : 1;
    const Sp<Real> &S = A.sp[si];
    const int64_t i = (tile - (si ? T0 : 0)) * TILE + (sl % TILE);
    if (i >= (si ? n1 : n0)) return;
    Real *d = pf + (size_t)b * NV * TILE + t;
    const Real *src[12] = {S.x, S.y, S.z, S.px, S.py, S.pz, S.ex, S.ey, S.ez, S.bx, S.by, S.bz};
#pragma unroll
    for (int c = 0; c < NV; ++c) cp_async<sizeof(Real)>(d + c * TILE, src[c] + i);
    cp_async<8>(pf_id + b * TILE + t, S.id + i);
  };
  const int64_t stride = (int64_t)gridDim.x * TILE;
  int buf = 0;
  int64_t slot = blockIdx.x * (int64_t)TILE + threadIdx.x;
  if (slot < nslots) prefetch(slot, 0);
  cp_async_commit();
  // nslots is a multiple of TILE: every lane of a warp runs the same iterations
  for (; slot < nslots; slot += stride, buf ^= 1) {
    if (slot + stride < nslots) prefetch(slot + stride, buf ^ 1);
    cp_async_commit();
    cp_async_wait<1>();  // this slot's copies have landed
    const int64_t tile = slot / TILE;
    const int si = tile < T0 ? 0 : 1;
    const Sp<Real> &S = A.sp[si];
    const int64_t i = (tile - (si ? T0 : 0)) * TILE + (slot % TILE);
    uint8_t flag = 0;
    Real x = 0, y = 0, z = 0, px = 0, py = 0, pz = 0;
    Real E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
    uint64_t pid = 0;
    if (i < (si ? n1 : n0)) {
      const Real *v = pf + (size_t)buf * NV * TILE + t;
      x = v[0]; y = v[TILE]; z = v[2 * TILE];
      px = v[3 * TILE]; py = v[4 * TILE]; pz = v[5 * TILE];
      if (FM == FM_PER_PARTICLE) {
        E[0] = v[6 * TILE]; E[1] = v[7 * TILE]; E[2] = v[8 * TILE];
        B[0] = v[9 * TILE]; B[1] = v[10 * TILE]; B[2] = v[11 * TILE];
      } else {
        get_fields<Real, FM>(S, A.f, i, x, y, z, E, B);
      }
      pid = pf_id[buf * TILE + t];
      Real g;
      if (MODE != MODE_EMIT) {
        g = boris(px, py, pz, E, B, S.q, dt);
        Real ig = r_div(dt, g);
        x += px * ig; y += py * ig; z += pz * ig;
      } else {
        g = m_sqrt((Real)1 + px * px + py * py + pz * pz);
      }
      if (!(g < (Real)1e30)) {
        tl.status |= QED_STATUS_NONFINITE;
      } else {
        Real chi = chi_lepton(px, py, pz, g, E[0], E[1], E[2], B[0], B[1], B[2], inv_aS);
        Tally t0;
        t0.clear();
        RateOut<Real> ro = photon_rate(sR, sF, A.T, A.C, chi, g, t0);
        const Real wdt = ro.W * dt;
        if (A.C.generator != GEN_METHOD_I) {
          // Methods II/III: P_cum += W Dt; an event when 1 - exp(-P_cum) > r3
          // (II) or P_cum > r3 (III); r3 is word 3 of the emission draw when
          // not drawn yet.  The emission itself (and the new P_cum, r3) is the
          // counting pass's, as a one-sub-step particle with an event.
          const U4 r = draw(A.C, pid, step_, 0, STREAM_EMIT);
          Real r3 = S.od_r[i];
          const bool fresh = !(r3 > (Real)0);
          if (fresh) r3 = unif<Real>(r.w);
          const Real P = S.od_p[i] + wdt;
          const bool ev = A.C.generator == GEN_METHOD_II ? -m_expm1(-P) > r3 : P > r3;
          if (ev) {
            flag = 1;
          } else {
            S.od_p[i] = P;
            if (fresh) S.od_r[i] = r3;
          }
        } else if (wdt > wdt_max) {
          // classes by sub-step count N = ceil(W Dt / wdt_max): 2: N <= 3, 3: N <= 7,
          // 4: N <= 15, 5: N >= 16 (lanes of a warp then do similar amounts of work)
          const Real q = r_div(wdt, wdt_max);
          flag = q <= (Real)3 ? 2 : (q <= (Real)7 ? 3 : (q <= (Real)15 ? 4 : 5));
        } else {
          U4 r = draw(A.C, pid, step_, 0, STREAM_EMIT);
          if (wdt > unif<Real>(r.x)) flag = 1;  // one sub-step with an event
        }
        if (flag == 0) {
          tl.status |= t0.status;
          tl.domain += t0.domain;
          tl.substeps += 1;
          if (MODE != MODE_EMIT) {
            S.x[i] = x; S.y[i] = y; S.z[i] = z;
            S.px[i] = px; S.py[i] = py; S.pz[i] = pz;
          }
        }
      }
    }
    A.heavy_flags[slot] = flag;
    // stage the pushed state of the flagged particles (warp-collective)
    const unsigned m = __ballot_sync(0xFFFFFFFFu, flag != 0);
    if (m) {
      const uint32_t cm = __popc(m);
      if (batch_used + cm > STAGE_BATCH) {
        uint32_t nb = 0;
        if (lane == 0) nb = atomicAdd(A.stage_n, STAGE_BATCH);
        batch_base = __shfl_sync(0xFFFFFFFFu, nb, 0);
        batch_used = 0;
      }
      if (flag) {
        const uint64_t pos = (uint64_t)batch_base + batch_used + __popc(m & ((1u << lane) - 1u));
        int32_t sidx = -1;
        if (pos < (uint64_t)A.stage_cap) {
          sidx = (int32_t)pos;
          Stage<Real> r;
          r.p[0] = px; r.p[1] = py; r.p[2] = pz;
          r.e[0] = E[0]; r.e[1] = E[1]; r.e[2] = E[2];
          r.b[0] = B[0]; r.b[1] = B[1]; r.b[2] = B[2];
          r.id_lo = (uint32_t)pid; r.id_hi = (uint32_t)(pid >> 32);
          r.w = S.w[i];
          r.x[0] = x; r.x[1] = y; r.x[2] = z;
          r.slot = (uint32_t)slot;
          const uint4 *src = reinterpret_cast<const uint4 *>(&r);
          uint4 *dst = reinterpret_cast<uint4 *>(A.stage + pos);
#pragma unroll
          for (int q = 0; q < (int)(sizeof(Stage<Real>) / 16); ++q) dst[q] = src[q];
          if (S.tag) A.stage_tag[pos] = S.tag[i];
          // the later passes read the staged copy; the pushed position and
          // momentum go to the arrays now, with the rest of the tile
          if (MODE != MODE_EMIT) {
            S.x[i] = x; S.y[i] = y; S.z[i] = z;
            S.px[i] = px; S.py[i] = py; S.pz[i] = pz;
          }
        }
        A.stage_idx[slot] = sidx;
      }
      batch_used += cm;
    }
  }
  cp_async_wait<0>();
  tally_flush(&bt, tl);
  __syncthreads();
  block_tally_commit(&bt, A.o.cnt, 0);
}

// ---------------------------------------------------------------------------
// Emission passes over the class list: every lepton the streaming pass could
// not finish (an event possible, or N > 1 by the rate bound).  The work is
// split so that no emission chain ever waits on another:
//   counting pass: the exact rate (with the xi_min cut) and N, then the
//     particle's Method I chain -- per sub-step one Philox draw, on an event
//     kappa from r2, ln delta from the inverse table (or the learned sampler
//     for N = 1), xi (Eq. 7) and the recoil -- writing only the number of
//     photons, the final gamma and the first REC emission records (photon
//     energy, sub-step index).  Particles are independent: no scan, no order.
//   scan: an in-place exclusive scan of the counts (one pass, decoupled
//     look-back over 4096-entry tiles of uniform cost) gives every particle
//     its first photon slot.
//   writing pass: the photons of each particle, from its records -- or, for a
//     particle with more than REC photons, from a replay of its chain -- and
//     its final momentum.
// Within a warp the chain is split into a scan phase (each lane draws until
// its next event) and an emission phase that the lanes with an event execute
// together, so lanes of different event counts stay converged.
// ---------------------------------------------------------------------------
constexpr int REC = SUB_REC;
// Work scheduling of the counting pass: a lane is idle (no particle), scanning
// (drawing sub-steps) or pending (an event found, its emission not yet done).
enum { LS_IDLE = 0, LS_SCAN = 1, LS_PEND = 2 };
constexpr int CNT_CHUNK = 64;       // entries per queue chunk of a warp
// An emission round waits for A.emit_lanes lanes with an event, a refill
// round for CNT_MIN_INIT idle lanes; a scanning round draws A.scan_draws
// sub-steps per lane.
constexpr int CNT_MIN_INIT = 20;

// A class-list entry's particle after the push.  Entry e >= 0 is staging
// record e (written by the streaming pass, which has also stored the pushed
// position and momentum); e < 0 is slot -e-1, a particle the staging area had
// no room for, gathered and pushed again from its unchanged stored state.
template <class Real> struct Entry {
  Real x, y, z, px, py, pz, g, w;
  Real E[3], B[3];
  uint64_t id;
  uint32_t tag;
  int64_t i;     // index in species si
  int si;
  bool staged;
};

template <class Real, int FM, int MODE>
__device__ __forceinline__ void load_entry(const LeptonArgs<Real> &A, int32_t e, int64_t T0,
                                           Real dt, Entry<Real> &P) {
  int64_t slot;
  P.staged = e >= 0;
  if (P.staged) {
    Stage<Real> r;
    const uint4 *src = reinterpret_cast<const uint4 *>(A.stage + e);
    uint4 *dst = reinterpret_cast<uint4 *>(&r);
#pragma unroll
    for (int q = 0; q < (int)(sizeof(Stage<Real>) / 16); ++q) dst[q] = __ldcs(src + q);
    P.px = r.p[0]; P.py = r.p[1]; P.pz = r.p[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) { P.E[c] = r.e[c]; P.B[c] = r.b[c]; }
    P.id = (uint64_t)r.id_lo | ((uint64_t)r.id_hi << 32);
    P.w = r.w;
    P.x = r.x[0]; P.y = r.x[1]; P.z = r.x[2];
    slot = r.slot;
  } else {
    slot = -(int64_t)e - 1;
  }
  const int64_t tile = slot / TILE;
  P.si = tile < T0 ? 0 : 1;
  P.i = (tile - (P.si ? T0 : 0)) * TILE + (slot % TILE);
  const Sp<Real> &S = A.sp[P.si];
  if (P.staged) {
    P.tag = S.tag ? A.stage_tag[e] : 0u;
    P.g = m_sqrt((Real)1 + P.px * P.px + P.py * P.py + P.pz * P.pz);
    return;
  }
  const int64_t i = P.i;
  P.x = S.x[i]; P.y = S.y[i]; P.z = S.z[i];
  P.px = S.px[i]; P.py = S.py[i]; P.pz = S.pz[i];
  get_fields<Real, FM>(S, A.f, i, P.x, P.y, P.z, P.E, P.B);
  P.id = S.id[i];
  P.w = S.w[i];
  P.tag = S.tag ? S.tag[i] : 0u;
  if (MODE != MODE_EMIT) {
    P.g = boris(P.px, P.py, P.pz, P.E, P.B, S.q, dt);
    Real ig = r_div(dt, P.g);
    P.x += P.px * ig; P.y += P.py * ig; P.z += P.pz * ig;
  } else {
    P.g = m_sqrt((Real)1 + P.px * P.px + P.py * P.py + P.pz * P.pz);
  }
}

// Final state of an entry after its emissions (final gamma g, unit direction
// n): a staged particle already has its pushed position stored.
template <class Real, int MODE>
__device__ __forceinline__ void store_entry(const LeptonArgs<Real> &A, const Entry<Real> &P,
                                            Real g, Real nx, Real ny, Real nz) {
  const Sp<Real> &S = A.sp[P.si];
  const int64_t i = P.i;
  const Real pm = m_sqrt((g - (Real)1) * (g + (Real)1));
  if (MODE != MODE_EMIT && !P.staged) { S.x[i] = P.x; S.y[i] = P.y; S.z[i] = P.z; }
  S.px[i] = pm * nx; S.py[i] = pm * ny; S.pz[i] = pm * nz;
}

template <class Real>
__device__ __forceinline__ void unit_dir(const Entry<Real> &P, Real &nx, Real &ny, Real &nz) {
  nx = ny = nz = 0;
  const Real pm = m_sqrt(P.px * P.px + P.py * P.py + P.pz * P.pz);
  if (pm > (Real)0) { Real ip = (Real)1 / pm; nx = P.px * ip; ny = P.py * ip; nz = P.pz * ip; }
}

// Sub-step count of a particle (Method I: N = max(1, ceil(W Dt / wdt_max))).
template <class Real>
__device__ __forceinline__ int64_t substep_count(const Consts &C, Real W, Real dt, Real wdt_max,
                                                 uint32_t &status) {
  const Real wdt = W * dt;
  if (!(wdt > wdt_max)) return 1;
  Real nn = m_ceil(wdt / wdt_max);
  if (nn > (Real)C.max_substeps) {
    nn = (Real)C.max_substeps;
    status |= QED_STATUS_SUBSTEPS;
  }
  return (int64_t)nn;
}

template <class Real, int FM, int MODE, bool MLP>
__global__ void __launch_bounds__(TILE, sizeof(Real) == 4 && !MLP ? 3 : 2) k_substep_count(LeptonArgs<Real> A) {
  const int64_t step_ = A.d_step ? *A.d_step : A.step;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kSmem = sizeof(Real) == 4;
  Real *sR = kSmem ? reinterpret_cast<Real *>(smem_raw) : const_cast<Real *>(A.T.R);
  Real *sF = kSmem ? sR + A.T.gl.n : const_cast<Real *>(A.T.F);
  // learned sampler image after the tables (FP32 contexts only)
  uint32_t *s_frag = reinterpret_cast<uint32_t *>(
      smem_raw + (kSmem ? (((size_t)A.T.gl.n * (1 + A.T.gy.n) * sizeof(Real) + 15) & ~(size_t)15) : 0));
  float *s_fw = reinterpret_cast<float *>(s_frag + MLP_FRAG_WORDS);
  constexpr bool use_mlp = kSmem && MLP;
  if (use_mlp) mlp_stage(s_frag, s_fw, A.mlp_frag, A.mlp_w);
  __shared__ long long s_meta[4];
  __shared__ BlockTally bt;
  if (kSmem) {
    load_tables_smem(sR, A.T.R, A.T.gl.n);
    load_tables_smem(sF, A.T.F, A.T.gl.n * A.T.gy.n);
  }
  block_tally_init(&bt);
  if (threadIdx.x == 0) {
    s_meta[0] = *(volatile int64_t *)A.sp[0].d_n;
    s_meta[1] = 0;  // the whole class list
    s_meta[2] = A.cls_off[NCLS];
  }
  __syncthreads();
  const int64_t T0 = (s_meta[0] + TILE - 1) / TILE;
  const int64_t begin = s_meta[1], nh = s_meta[2] - s_meta[1];
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const Real inv_aS = sel<Real>(A.C.inv_aS, A.C.f_inv_aS);
  const Real dt = sel<Real>(A.C.dt, A.C.f_dt);
  const Real wdt_max = sel<Real>(A.C.wdt_max, A.C.f_wdt_max);
  const int64_t rc = A.rec_cap;
  Tally tl;
  tl.clear();
  // This warp's queue: chunks w, w + W, w + 2W, ... of CNT_CHUNK entries,
  // counted from the end of the list (the heaviest classes first).
  const int64_t W = (int64_t)gridDim.x * (TILE / 32);
  const int64_t w = blockIdx.x * (int64_t)(TILE / 32) + (threadIdx.x >> 5);
  const int64_t nchunks = (nh + CNT_CHUNK - 1) / CNT_CHUNK;
  const int64_t qend = w < nchunks ? ((nchunks - 1 - w) / W + 1) * CNT_CHUNK : 0;
  int64_t next = 0;  // queue position (warp-uniform)
  // lane state
  int state = LS_IDLE;
  int64_t h = 0, N = 0, k = 0;
  uint32_t cnt = 0, wy = 0;
  Real px = 0, py = 0, pz = 1, g = 1, chi = 0, dts = 0, nx = 0, ny = 0, nz = 0;
  Real E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
  uint64_t pid = 0;
  RateOut<Real> ro{(Real)0, (Real)-1e30, (Real)0};
  // Methods II/III: the particle's species, index and the word for its next r3
  int psi = 0;
  int64_t pi = 0;
  uint32_t w3 = 0;
  auto finish = [&]() {
    tl.events += cnt;
    A.sub_cnt[h] = cnt;
    if (h < rc) A.sub_gf[h] = g;
    if (A.C.generator != GEN_METHOD_I) {  // P_cum restarts with a fresh r3 (word 2)
      A.sp[psi].od_p[pi] = (Real)0;
      A.sp[psi].od_r[pi] = unif<Real>(w3);
    }
    state = LS_IDLE;
  };
  for (;;) {
    const unsigned idle = __ballot_sync(0xFFFFFFFFu, state == LS_IDLE);
    const unsigned pend = __ballot_sync(0xFFFFFFFFu, state == LS_PEND);
    const unsigned scan = __ballot_sync(0xFFFFFFFFu, state == LS_SCAN);
    const bool more = next < qend;
    // one phase per round, run by every lane in that state: emission once
    // enough lanes wait for it, refills once enough lanes are idle, else
    // draws; the fall-backs guarantee progress
    int phase;
    if (__popc(pend) >= A.emit_lanes) phase = LS_PEND;
    else if (more && __popc(idle) >= CNT_MIN_INIT) phase = LS_IDLE;
    else if (scan) phase = LS_SCAN;
    else if (pend) phase = LS_PEND;
    else if (more && idle) phase = LS_IDLE;
    else break;
    if (phase == LS_IDLE) {
      // refill: the idle lanes take the next queue positions, in lane order
      if (state == LS_IDLE) {
        const int64_t q = next + __popc(idle & lt_mask);
        const int64_t hr = q < qend ? (w + (q / CNT_CHUNK) * W) * CNT_CHUNK + (q % CNT_CHUNK) : nh;
        if (hr < nh) {
          h = nh - 1 - hr;
          Entry<Real> P;
          load_entry<Real, FM, MODE>(A, A.heavy_list[begin + h], T0, dt, P);
          px = P.px; py = P.py; pz = P.pz; g = P.g;
#pragma unroll
          for (int c = 0; c < 3; ++c) { E[c] = P.E[c]; B[c] = P.B[c]; }
          pid = P.id;
          unit_dir(P, nx, ny, nz);
          chi = chi_lepton(px, py, pz, g, E[0], E[1], E[2], B[0], B[1], B[2], inv_aS);
          ro = photon_rate(sR, sF, A.T, A.C, chi, g, tl);
          k = 0;
          cnt = 0;
          if (A.C.generator != GEN_METHOD_I) {
            // Methods II/III: the streaming pass found the event; one photon,
            // its xi from word 1 of the step's emission draw
            const U4 r = draw(A.C, pid, step_, 0, STREAM_EMIT);
            N = 1;
            dts = dt;
            wy = r.y;
            w3 = r.z;
            psi = P.si;
            pi = P.i;
            tl.substeps += 1;
            state = LS_PEND;
          } else {
            N = substep_count(A.C, ro.W, dt, wdt_max, tl.status);
            tl.substeps += N;
            dts = dt / (Real)N;
            state = LS_SCAN;
          }
        }
      }
      next += __popc(idle);
    } else if (phase == LS_SCAN) {
      // Method I draws until an event or the last sub-step; one Philox call
      // gives the words of two sub-steps (2j and 2j+1)
      if (state == LS_SCAN) {
        const Real thr = ro.W * dts;
        for (int s = 0; s < A.scan_draws; s += 2) {
          const U4 r = draw(A.C, pid, step_, k >> 1, STREAM_EMIT);
          if (!(k & 1)) {
            if (thr > unif<Real>(r.x)) { wy = r.y; state = LS_PEND; break; }
            if (++k >= N) { finish(); break; }
          }
          if (thr > unif<Real>(r.z)) { wy = r.w; state = LS_PEND; break; }
          if (++k >= N) { finish(); break; }
        }
      }
    } else {
      // emission, by every lane with an event: kappa from r2 (Eq. 7), then
      // ln delta from the inverse table -- or, for a particle with N = 1 in a
      // context with the learned sampler, from the network (a warp-collective
      // call, made by every lane, only in rounds where some lane needs it)
      const bool ev = state == LS_PEND;
      const Real kap = ev ? photon_kappa(ro.kmin, unif<Real>(wy), unif<Real>(~wy)) : (Real)0;
      Real Y = (Real)0;
      bool in_mlp = false;
      if (use_mlp && __any_sync(0xFFFFFFFFu, ev && N == 1)) {
        const float lchi = chi > (Real)0 ? (float)m_log(chi) : MLP_L_LO - 1.0f;
        in_mlp = ev && N == 1 && lchi >= MLP_L_LO && lchi <= MLP_L_HI && (float)kap >= MLP_K_LO &&
                 (float)kap <= MLP_K_HI;
        const float zz = mlp_infer_warp(s_frag, s_fw, (lchi - MLP_LC) / MLP_LS,
                                        ((float)kap - MLP_KC) / MLP_KS);
        Y = (Real)(zz + mlp_baseline((float)kap));
      }
      if (ev) {
        if (!in_mlp) Y = photon_lndelta_table(A.T.Y, A.T, ro.l, kap, tl);
        XiOut<Real> xo = xi_from_lndelta(chi, Y);
        Real g2 = g * xo.omxi, eph = g * xo.xi;
        if (g2 < (Real)1) { g2 = (Real)1; eph = g - (Real)1; }
        if (cnt < REC && h < rc) {
          A.rec_e[cnt * rc + h] = eph;
          A.rec_k[cnt * rc + h] = (uint32_t)k;
        }
        ++cnt;
        int b = spec_bin(A.C, eph);
        {  // one shared atomic per distinct bin among the emitting lanes
          const unsigned em = __activemask();
          const unsigned same = __match_any_sync(em, b);
          if (b >= 0 && lane == __ffs(same) - 1) atomicAdd(&bt.hist[b], (unsigned long long)__popc(same));
        }
        Real pm2 = m_sqrt((g2 - (Real)1) * (g2 + (Real)1));
        px = pm2 * nx; py = pm2 * ny; pz = pm2 * nz;
        g = g2;
        if (++k >= N) {
          finish();
        } else {  // the rate for the remaining sub-steps
          chi = chi_lepton(px, py, pz, g, E[0], E[1], E[2], B[0], B[1], B[2], inv_aS);
          ro = photon_rate(sR, sF, A.T, A.C, chi, g, tl);
          state = LS_SCAN;
        }
      }
    }
  }
  tally_flush(&bt, tl);
  __syncthreads();
  block_tally_commit(&bt, A.o.cnt, 0);
}

// Writing pass, warp-cooperative: a warp takes 32 consecutive entries; each
// lane stores its own particle's final state, and then the warp's photons are
// written by consecutive lanes -- one photon per lane, its parent's data
// fetched by shuffles -- so the 15 per-photon stores (state, id, alive flag,
// fields) are coalesced and every lane has a photon to write.  Particles whose
// photons are not all recorded are listed for the replay launch
// (k_substep_replay).
template <class Real, int FM, int MODE>
__global__ void __launch_bounds__(TILE, sizeof(Real) == 4 ? 4 : 2) k_substep_write_coop(LeptonArgs<Real> A) {
  const int64_t step_ = A.d_step ? *A.d_step : A.step;
  __shared__ uint8_t s_parent[TILE / 32][32 * REC];  // warp photon -> parent lane
  __shared__ long long s_meta[4];
  __shared__ BlockTally bt;
  block_tally_init(&bt);
  if (threadIdx.x == 0) {
    s_meta[0] = *(volatile int64_t *)A.sp[0].d_n;
    s_meta[1] = A.cls_off[NCLS];
    s_meta[2] = A.sub_meta[0];  // photons of all entries
    s_meta[3] = A.sub_meta[1];  // photon count before them
  }
  __syncthreads();
  const int64_t T0 = (s_meta[0] + TILE - 1) / TILE;
  const int64_t nh = s_meta[1];
  const uint32_t total = (uint32_t)s_meta[2];
  const int64_t nph = s_meta[3];
  const Real dt = sel<Real>(A.C.dt, A.C.f_dt);
  const int64_t rc = A.rec_cap;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint8_t *par = s_parent[wid];
  Tally tl;
  tl.clear();
  const int64_t nwarps = (int64_t)gridDim.x * (TILE / 32);
  for (int64_t wb = (blockIdx.x * (int64_t)(TILE / 32) + wid) * 32; wb < nh; wb += nwarps * 32) {
    const int64_t h = wb + lane;
    const bool act = h < nh;
    uint32_t off = 0, cnt = 0;
    int32_t e = 0;
    if (act) {
      off = A.sub_cnt[h];  // exclusive prefix of the counts now
      cnt = (h + 1 < nh ? A.sub_cnt[h + 1] : total) - off;
      e = A.heavy_list[h];
    }
    const bool rep = act && cnt > 0 && (cnt > REC || h >= rc);
    if (rep) A.replay_list[atomicAdd(A.replay_n, 1u)] = (int32_t)h;
    const uint32_t mine = (act && !rep) ? cnt : 0u;  // photons this lane's entry gives the warp
    // the particle: staged with no photon needs nothing (the streaming pass
    // stored it); otherwise its final state is stored here
    Entry<Real> P;
    P.x = P.y = P.z = P.px = P.py = P.w = (Real)0;
    P.pz = P.g = (Real)1;
#pragma unroll
    for (int c = 0; c < 3; ++c) { P.E[c] = (Real)0; P.B[c] = (Real)0; }
    P.id = 0;
    P.tag = 0;
    Real nx = 0, ny = 0, nz = 0;
    const bool need = act && !rep && (cnt > 0 || e < 0);
    if (need) {
      Real gfin = (Real)0;
      if (cnt > 0) gfin = A.sub_gf[h];
      load_entry<Real, FM, MODE>(A, e, T0, dt, P);
      unit_dir(P, nx, ny, nz);
      store_entry<Real, MODE>(A, P, cnt > 0 ? gfin : P.g, nx, ny, nz);
    }
    // the warp's photons, in entry order
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    const uint32_t excl = incl - mine;
    const uint32_t T = __shfl_sync(0xFFFFFFFFu, incl, 31);
    for (uint32_t j = 0; j < mine; ++j) par[excl + j] = (uint8_t)lane;
    __syncwarp();
    for (uint32_t q0 = 0; q0 < T; q0 += 32) {
      const uint32_t q = q0 + lane;
      const bool valid = q < T;
      const int L = valid ? par[q] : 0;
      // the parent's data, by shuffles (every lane takes part)
      const Real x = __shfl_sync(0xFFFFFFFFu, P.x, L), y = __shfl_sync(0xFFFFFFFFu, P.y, L),
                 z = __shfl_sync(0xFFFFFFFFu, P.z, L);
      const Real ux = __shfl_sync(0xFFFFFFFFu, nx, L), uy = __shfl_sync(0xFFFFFFFFu, ny, L),
                 uz = __shfl_sync(0xFFFFFFFFu, nz, L);
      const Real w = __shfl_sync(0xFFFFFFFFu, P.w, L);
      Real E[3], B[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        E[c] = __shfl_sync(0xFFFFFFFFu, P.E[c], L);
        B[c] = __shfl_sync(0xFFFFFFFFu, P.B[c], L);
      }
      const uint64_t pid = (uint64_t)__shfl_sync(0xFFFFFFFFu, (unsigned long long)P.id, L);
      const uint32_t ptag = __shfl_sync(0xFFFFFFFFu, P.tag, L);
      const uint32_t poff = __shfl_sync(0xFFFFFFFFu, off, L);
      const uint32_t pex = __shfl_sync(0xFFFFFFFFu, excl, L);
      const int64_t ph = wb + L;
      if (!valid) continue;
      const uint32_t j = q - pex;  // the parent's j-th photon
      const Real eph = A.rec_e[j * rc + ph];
      const int64_t kk = A.rec_k[j * rc + ph];
      const int64_t out = nph + (int64_t)poff + j;
      if (out >= A.ph.cap) {
        tl.dropped += 1;
        tl.status |= QED_STATUS_CAPACITY;
        continue;
      }
      const U4 cid = draw(A.C, pid, step_, kk, STREAM_PHOTON_ID);
      write_child(A.ph, out, x, y, z, eph * ux, eph * uy, eph * uz, w,
                  (uint64_t)cid.x | ((uint64_t)cid.y << 32), E, B, ptag);
    }
    __syncwarp();  // par is rewritten by the next window
  }
  tally_flush(&bt, tl);
  __syncthreads();
  block_tally_commit(&bt, A.o.cnt, 0);
}

// Exclusive scan, in place, of the sub-step entries' photon counts (single
// pass, decoupled look-back over 4096-entry tiles).  The total and the photon
// count at launch go to sub_meta[0] and sub_meta[1]; the last tile publishes
// the new photon count.
struct SubScanArgs {
  uint32_t *cnt;
  unsigned int *replay_n;  // reset here for the writing pass
  const int64_t *n_entries;
  int64_t *sub_meta;       // [0] total, [1] count of out1 before, [2] count of out2 before
  int64_t *out1_n, *out2_n;  // species counts to advance by the total (out2 optional)
  int64_t out1_cap, out2_cap;
  Out o;
};
constexpr int SCAN_ITEMS = 16;

__global__ void __launch_bounds__(TILE) k_sub_scan(SubScanArgs A) {
  __shared__ uint32_t scan_sm[33];
  __shared__ long long s_meta[6];
  if (threadIdx.x == 0) {
    s_meta[2] = *(volatile const int64_t *)A.n_entries;
    s_meta[3] = *(volatile int64_t *)A.out1_n;
    s_meta[4] = (long long)A.o.scan.sync[2];
    s_meta[5] = A.out2_n ? *(volatile int64_t *)A.out2_n : 0;
  }
  __syncthreads();
  const int64_t nh = s_meta[2], nph = s_meta[3], n2 = s_meta[5];
  const uint32_t epoch = (uint32_t)s_meta[4];
  const int64_t per_tile = (int64_t)TILE * SCAN_ITEMS;
  const int64_t ntiles = (nh + per_tile - 1) / per_tile;
  uint32_t status = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *A.replay_n = 0u;
    if (ntiles == 0) {
      A.sub_meta[0] = 0;
      A.sub_meta[1] = nph;
      A.sub_meta[2] = n2;
    }
  }
  for (;;) {
    if (threadIdx.x == 0) s_meta[0] = (long long)atomicAdd(&A.o.scan.sync[0], 1u);
    __syncthreads();
    const int64_t t = s_meta[0];
    __syncthreads();
    if (t >= ntiles) break;
    const int64_t first = t * per_tile + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
      v[j] = first + j < nh ? A.cnt[first + j] : 0u;
      sum += v[j];
    }
    const uint32_t excl = block_excl_scan(sum, scan_sm);
    const uint32_t agg = scan_sm[32];
    if (threadIdx.x < 32) {
      const uint32_t pre = lookback_warp(A.o.scan, t, epoch, agg, status);
      if (threadIdx.x == 0) {
        s_meta[1] = pre;
        if (t == ntiles - 1) {
          const int64_t tot = (int64_t)pre + agg;
          A.sub_meta[0] = tot;
          A.sub_meta[1] = nph;
          A.sub_meta[2] = n2;
          *A.out1_n = nph + tot < A.out1_cap ? nph + tot : A.out1_cap;
          if (A.out2_n) *A.out2_n = n2 + tot < A.out2_cap ? n2 + tot : A.out2_cap;
        }
      }
    }
    __syncthreads();
    uint32_t run = (uint32_t)s_meta[1] + excl;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
      if (first + j < nh) A.cnt[first + j] = run;
      run += v[j];
    }
  }
  if (threadIdx.x == 0 && status) atomicOr(&A.o.cnt->status, status);
  launch_epilogue(A.o.scan, epoch);
}

// Replay launch of the writing pass: the particles k_substep_write_coop listed
// (more than REC photons, or past the record capacity, both rare) redo their
// emission chains -- same draws, same tables -- and write their photons and
// final momenta.  It is separate so that the common case carries neither the
// tables nor the chain's registers, and dense, so that the rare long replays
// share warps.
template <class Real, int FM, int MODE>
__global__ void __launch_bounds__(TILE, 2) k_substep_replay(LeptonArgs<Real> A) {
  const int64_t step_ = A.d_step ? *A.d_step : A.step;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kSmem = sizeof(Real) == 4;
  Real *sR = kSmem ? reinterpret_cast<Real *>(smem_raw) : const_cast<Real *>(A.T.R);
  Real *sF = kSmem ? sR + A.T.gl.n : const_cast<Real *>(A.T.F);
  __shared__ long long s_meta[4];
  __shared__ BlockTally bt;
  // a block with nothing to replay leaves before staging the tables
  const int64_t n_iter = (int64_t)*(volatile unsigned int *)A.replay_n;
  if ((int64_t)blockIdx.x * TILE >= n_iter) return;
  if (kSmem) {
    load_tables_smem(sR, A.T.R, A.T.gl.n);
    load_tables_smem(sF, A.T.F, A.T.gl.n * A.T.gy.n);
  }
  block_tally_init(&bt);
  if (threadIdx.x == 0) {
    s_meta[0] = *(volatile int64_t *)A.sp[0].d_n;
    s_meta[1] = A.cls_off[NCLS];
    s_meta[2] = A.sub_meta[0];  // photons of all entries
    s_meta[3] = A.sub_meta[1];  // photon count before them
  }
  __syncthreads();
  const int64_t T0 = (s_meta[0] + TILE - 1) / TILE;
  const int64_t nh = s_meta[1];
  const uint32_t total = (uint32_t)s_meta[2];
  const int64_t nph = s_meta[3];
  const Real inv_aS = sel<Real>(A.C.inv_aS, A.C.f_inv_aS);
  const Real dt = sel<Real>(A.C.dt, A.C.f_dt);
  const Real wdt_max = sel<Real>(A.C.wdt_max, A.C.f_wdt_max);
  Tally tl;
  tl.clear();
  for (int64_t q = blockIdx.x * (int64_t)TILE + threadIdx.x; q < n_iter; q += (int64_t)gridDim.x * TILE) {
    const int64_t h = (int64_t)A.replay_list[q];
    // sub_cnt holds the exclusive prefix of the counts now
    const uint32_t off = A.sub_cnt[h];
    const uint32_t cnt = (h + 1 < nh ? A.sub_cnt[h + 1] : total) - off;
    const int32_t e = A.heavy_list[h];
    const int64_t out0 = nph + (int64_t)off;
    Entry<Real> P;
    load_entry<Real, FM, MODE>(A, e, T0, dt, P);
    Real nx, ny, nz;
    unit_dir(P, nx, ny, nz);
    Real g = P.g;
    auto put = [&](uint32_t j, Real eph, int64_t kk) {
      const int64_t out = out0 + j;
      if (out >= A.ph.cap) {
        tl.dropped += 1;
        tl.status |= QED_STATUS_CAPACITY;
        return;
      }
      U4 cid = draw(A.C, P.id, step_, kk, STREAM_PHOTON_ID);
      write_child(A.ph, out, P.x, P.y, P.z, eph * nx, eph * ny, eph * nz, P.w,
                  (uint64_t)cid.x | ((uint64_t)cid.y << 32), P.E, P.B, P.tag);
    };
    // the chain again (its counters went to the counting pass's tally)
    Tally dummy;
    dummy.clear();
    const Real *E = P.E, *B = P.B;
    Real chi = chi_lepton(P.px, P.py, P.pz, g, E[0], E[1], E[2], B[0], B[1], B[2], inv_aS);
    RateOut<Real> ro = photon_rate(sR, sF, A.T, A.C, chi, g, dummy);
    const bool forced = A.C.generator != GEN_METHOD_I;  // Methods II/III: one photon at k = 0
    const int64_t N = forced ? 1 : substep_count(A.C, ro.W, dt, wdt_max, dummy.status);
    const Real dts = dt / (Real)N;
    uint32_t j = 0;
    for (int64_t kk = 0; kk < N && j < cnt; ++kk) {
      const EmitWords r = emit_words(A.C, P.id, step_, kk);
      if (!forced && !(ro.W * dts > unif<Real>(r.r1))) continue;
      XiOut<Real> xo = photon_xi(A.T.Y, A.T, ro.l, chi, ro.kmin, unif<Real>(r.r2), unif<Real>(~r.r2), dummy);
      Real g2 = g * xo.omxi, eph = g * xo.xi;
      if (g2 < (Real)1) { g2 = (Real)1; eph = g - (Real)1; }
      put(j++, eph, kk);
      Real pm2 = m_sqrt((g2 - (Real)1) * (g2 + (Real)1));
      g = g2;
      chi = chi_lepton(pm2 * nx, pm2 * ny, pm2 * nz, g, E[0], E[1], E[2], B[0], B[1], B[2], inv_aS);
      ro = photon_rate(sR, sF, A.T, A.C, chi, g, dummy);
    }
    if (j != cnt) {  // the replay disagreed with the count: zero-energy photons fill the slots
      tl.status |= QED_STATUS_REPLAY;
      for (; j < cnt; ++j) put(j, (Real)0, 0);
    }
    store_entry<Real, MODE>(A, P, g, nx, ny, nz);
  }
  tally_flush(&bt, tl);
  __syncthreads();
  block_tally_commit(&bt, A.o.cnt, 0);
}

// ---------------------------------------------------------------------------
// Ordered list of the deferred (heavy) particles: stable compaction of the
// streaming pass's flags, one flag per slot (tile * TILE + lane).
// ---------------------------------------------------------------------------
struct HeavyListArgs {
  const uint8_t *flags;
  uint8_t want;  // flag value to collect
  const int32_t *stage_idx;  // if set: list the staging record (or -(slot + 1))
  int *list;
  int64_t *count;
  const int64_t *n0, *n1;  // species counts (size the streaming pass's slot range)
  Out o;
};

constexpr int LIST_ITEMS = 16;  // flags per thread (one 16-byte load)

__global__ void __launch_bounds__(TILE) k_heavy_list(HeavyListArgs A) {
  __shared__ uint32_t scan_sm[33];
  __shared__ long long s_meta[8];
  if (threadIdx.x == 0) {
    int64_t n0 = *(volatile const int64_t *)A.n0;
    int64_t n1 = A.n1 ? *(volatile const int64_t *)A.n1 : 0;
    s_meta[2] = ((n0 + TILE - 1) / TILE + (n1 + TILE - 1) / TILE) * TILE;  // flag slots
    s_meta[5] = (long long)A.o.scan.sync[2];
  }
  __syncthreads();
  const int64_t nslots = s_meta[2];
  const int64_t per_tile = (int64_t)TILE * LIST_ITEMS;
  const int64_t ntiles = (nslots + per_tile - 1) / per_tile;
  const uint32_t epoch = (uint32_t)s_meta[5];
  uint32_t status = 0;
  if (ntiles == 0 && blockIdx.x == 0 && threadIdx.x == 0) *A.count = 0;
  for (;;) {
    if (threadIdx.x == 0) s_meta[0] = (long long)atomicAdd(&A.o.scan.sync[0], 1u);
    __syncthreads();
    const int64_t t = s_meta[0];
    __syncthreads();
    if (t >= ntiles) break;
    const int64_t first = t * per_tile + (int64_t)threadIdx.x * LIST_ITEMS;
    uint4 raw = make_uint4(0, 0, 0, 0);
    if (first < nslots) raw = *reinterpret_cast<const uint4 *>(A.flags + first);
    const uint8_t *fl = reinterpret_cast<const uint8_t *>(&raw);
    uint32_t mask = 0;
#pragma unroll
    for (int j = 0; j < LIST_ITEMS; ++j)
      if (fl[j] == A.want && first + j < nslots) mask |= 1u << j;
    uint32_t cnt = __popc(mask);
    uint32_t excl = block_excl_scan(cnt, scan_sm);
    uint32_t agg = scan_sm[32];
    if (threadIdx.x < 32) {
      uint32_t pre = lookback_warp(A.o.scan, t, epoch, agg, status);
      if (threadIdx.x == 0) {
        s_meta[1] = pre;
        if (t == ntiles - 1) *A.count = (int64_t)pre + agg;
      }
    }
    __syncthreads();
    int64_t out = s_meta[1] + excl;
    while (mask) {
      int j = __ffs(mask) - 1;
      mask &= mask - 1;
      int v = (int)(first + j);
      if (A.stage_idx) {
        const int32_t sidx = A.stage_idx[first + j];
        v = sidx >= 0 ? sidx : -v - 1;
      }
      A.list[out++] = v;
    }
  }
  if (threadIdx.x == 0 && status) atomicOr(&A.o.cnt->status, status);
  launch_epilogue(A.o.scan, epoch);
}

// ---------------------------------------------------------------------------
// Class list of the streaming pass's flagged leptons: one ordered list,
// class-major (all class-1 slots in slot order, then class 2, ..., class 5),
// built by a count, a scan and a scatter pass -- no CTA waits on another.
// off[c - 1] is the first list position of class c and off[NCLS] the length.
// Flags are read 8 per thread (one 8-byte load), 2048 per chunk; a chunk's
// per-class counts (<= 2048 each) are packed 12 bits per class in a uint64.
// ---------------------------------------------------------------------------
constexpr int CLS_ITEMS = 8;
constexpr int CLS_CHUNK = TILE * CLS_ITEMS;
static_assert(CLS_CHUNK == CLS_CHUNK_FLAGS, "class-list chunk size");
constexpr int CLS_SCAN_THREADS = 1024;
constexpr int CLS_SCAN_PER_THREAD = 8;  // chunks per thread per round of the scan

struct ClassListArgs {
  const uint8_t *flags;
  const int64_t *n0, *n1;  // species counts (size the streaming pass's slot range)
  int *list;
  unsigned long long *chunk_cnt;  // [chunks] packed per-class counts
  uint32_t *chunk_off;            // [chunks][NCLS] first list position per class
  int64_t *off;                   // [NCLS + 1]
  const int32_t *stage_idx;       // [slot] staging record of a flagged slot (-1: none)
  unsigned int *stage_n;          // staging counter, reset by the scan for the next step
  qed_counters *cnt;              // deferred += list length
};

__device__ __forceinline__ int64_t cls_nslots(const ClassListArgs &A) {
  const int64_t n0 = *(volatile const int64_t *)A.n0;
  const int64_t n1 = A.n1 ? *(volatile const int64_t *)A.n1 : 0;
  return ((n0 + TILE - 1) / TILE + (n1 + TILE - 1) / TILE) * TILE;
}

// This thread's 8 flags of chunk c and their packed per-class counts.  The
// slot range is a multiple of TILE, so a group of 8 is all in or all out.
__device__ __forceinline__ unsigned long long cls_load(const ClassListArgs &A, int64_t c,
                                                       int64_t nslots, uint2 &raw) {
  const int64_t first = c * CLS_CHUNK + (int64_t)threadIdx.x * CLS_ITEMS;
  raw = make_uint2(0u, 0u);
  if (first < nslots) raw = *reinterpret_cast<const uint2 *>(A.flags + first);
  const uint8_t *fl = reinterpret_cast<const uint8_t *>(&raw);
  unsigned long long packed = 0;
#pragma unroll
  for (int j = 0; j < CLS_ITEMS; ++j)
    if (fl[j] >= 1 && fl[j] <= NCLS) packed += 1ull << (12 * (fl[j] - 1));
  return packed;
}

// Block-wide exclusive scan of a uint64 per thread; sm needs 33 words and
// receives the block total in sm[32].
__device__ __forceinline__ unsigned long long block_excl_scan64(unsigned long long v,
                                                               unsigned long long *sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) sm[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    unsigned long long w = lane < nw ? sm[lane] : 0ull, wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += u;
    }
    if (lane < nw) sm[lane] = wi - w;
    if (lane == nw - 1) sm[32] = wi;
  }
  __syncthreads();
  const unsigned long long r = sm[wid] + incl - v;
  __syncthreads();
  return r;
}

__device__ __forceinline__ uint32_t cls_field(unsigned long long p, int c) {
  return (uint32_t)(p >> (12 * c)) & 0xFFFu;
}

__global__ void __launch_bounds__(TILE) k_cls_count(ClassListArgs A) {
  __shared__ unsigned long long sm[33];
  const int64_t nslots = cls_nslots(A);
  const int64_t nchunks = (nslots + CLS_CHUNK - 1) / CLS_CHUNK;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    uint2 raw;
    const unsigned long long p = cls_load(A, c, nslots, raw);
    block_excl_scan64(p, sm);
    if (threadIdx.x == 0) A.chunk_cnt[c] = sm[32];
  }
}

// One CTA: class totals, class starts, and every chunk's per-class offset.
__global__ void __launch_bounds__(CLS_SCAN_THREADS) k_cls_scan(ClassListArgs A) {
  __shared__ unsigned long long tot[NCLS];
  __shared__ unsigned long long sm[33];
  __shared__ int64_t base[NCLS];
  const int64_t nslots = cls_nslots(A);
  const int64_t nchunks = (nslots + CLS_CHUNK - 1) / CLS_CHUNK;
  if (threadIdx.x < NCLS) tot[threadIdx.x] = 0;
  if (threadIdx.x == 0) *A.stage_n = 0u;  // the streaming pass of this step is done with it
  __syncthreads();
  unsigned long long mine[NCLS] = {0, 0, 0, 0, 0};
  for (int64_t c = threadIdx.x; c < nchunks; c += blockDim.x) {
    const unsigned long long p = A.chunk_cnt[c];
#pragma unroll
    for (int k = 0; k < NCLS; ++k) mine[k] += cls_field(p, k);
  }
#pragma unroll
  for (int k = 0; k < NCLS; ++k) {
    unsigned long long v = mine[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&tot[k], v);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t b = 0;
    for (int k = 0; k < NCLS; ++k) {
      base[k] = b;
      A.off[k] = b;
      b += (int64_t)tot[k];
    }
    A.off[NCLS] = b;
    if (b) atomicAdd(reinterpret_cast<unsigned long long *>(&A.cnt->deferred), (unsigned long long)b);
  }
  __syncthreads();
  // per-class running prefix over chunks; each round a thread takes
  // CLS_SCAN_PER_THREAD consecutive chunks.  A round's prefixes stay below
  // 2^25 per class (2048 * 8 * 1024), so two classes share a packed scan.
  int64_t carry[NCLS];
#pragma unroll
  for (int k = 0; k < NCLS; ++k) carry[k] = base[k];
  const int64_t per_round = (int64_t)blockDim.x * CLS_SCAN_PER_THREAD;
  for (int64_t r0 = 0; r0 < nchunks; r0 += per_round) {
    const int64_t c0 = r0 + (int64_t)threadIdx.x * CLS_SCAN_PER_THREAD;
    uint32_t t[NCLS + 1] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < CLS_SCAN_PER_THREAD; ++j) {
      const int64_t c = c0 + j;
      if (c < nchunks) {
        const unsigned long long p = A.chunk_cnt[c];
#pragma unroll
        for (int k = 0; k < NCLS; ++k) t[k] += cls_field(p, k);
      }
    }
    uint32_t run[NCLS + 1], rtot[NCLS + 1];
#pragma unroll
    for (int q = 0; q < (NCLS + 1) / 2; ++q) {
      const unsigned long long v = (unsigned long long)t[2 * q] | ((unsigned long long)t[2 * q + 1] << 32);
      const unsigned long long e = block_excl_scan64(v, sm), tt = sm[32];
      run[2 * q] = (uint32_t)e;
      run[2 * q + 1] = (uint32_t)(e >> 32);
      rtot[2 * q] = (uint32_t)tt;
      rtot[2 * q + 1] = (uint32_t)(tt >> 32);
    }
#pragma unroll
    for (int j = 0; j < CLS_SCAN_PER_THREAD; ++j) {
      const int64_t c = c0 + j;
      if (c < nchunks) {
        const unsigned long long p = A.chunk_cnt[c];
#pragma unroll
        for (int k = 0; k < NCLS; ++k) {
          A.chunk_off[c * NCLS + k] = (uint32_t)(carry[k] + run[k]);
          run[k] += cls_field(p, k);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NCLS; ++k) carry[k] += (int64_t)rtot[k];
  }
}

__global__ void __launch_bounds__(TILE) k_cls_scatter(ClassListArgs A) {
  __shared__ unsigned long long sm[33];
  const int64_t nslots = cls_nslots(A);
  const int64_t nchunks = (nslots + CLS_CHUNK - 1) / CLS_CHUNK;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    uint2 raw;
    const unsigned long long p = cls_load(A, c, nslots, raw);
    unsigned long long ex = block_excl_scan64(p, sm);
    if (!p) continue;
    const uint8_t *fl = reinterpret_cast<const uint8_t *>(&raw);
    const int64_t first = c * CLS_CHUNK + (int64_t)threadIdx.x * CLS_ITEMS;
#pragma unroll
    for (int j = 0; j < CLS_ITEMS; ++j) {
      const int k = (int)fl[j] - 1;
      if (k < 0 || k >= NCLS) continue;
      // list entry: the staging record, or -(slot + 1) for an unstaged slot
      const int32_t sidx = A.stage_idx[first + j];
      A.list[A.chunk_off[c * NCLS + k] + cls_field(ex, k)] = sidx >= 0 ? sidx : -(int32_t)(first + j) - 1;
      ex += 1ull << (12 * k);
    }
  }
}

// ---------------------------------------------------------------------------
// Photon kernel: push + Breit-Wheeler pairs
// ---------------------------------------------------------------------------
template <class Real> struct PhotonArgs {
  Sp<Real> ph, el, po;
  const int64_t *n_active;  // photons [0, *n_active) are processed
  Fld<Real> f;
  Consts C;
  Tables<Real> T;
  Out o;
  int64_t step;
  uint8_t *flags;       // streaming pass: 1 = redo in the ordered pass
  const int *list;      // ordered pass: staging record (>= 0) or -(index + 1)
  Stage<Real> *stage;   // pushed state of the flagged photons (streaming pass)
  uint32_t *stage_tag;
  int32_t *stage_idx;   // [index] staging record of a flagged photon, -1 if not staged
  unsigned int *stage_n;
  int64_t stage_cap;
  const int64_t *list_n;
  const int64_t *d_step;  // if set, the step index is read here (graph replay)
  uint32_t *sub_cnt;      // pairs per list entry, then their exclusive prefix
  const int64_t *sub_meta;  // [0] pairs in all, [1] electrons before, [2] positrons before
  Real *rec_e;            // [0][h] gamma_e, [1][h] gamma_p of entry h's pair (h < rec_cap)
  uint32_t *rec_k;        // [h] its sub-step
  int64_t rec_cap;
};

// ---------------------------------------------------------------------------
// Streaming photon pass: ballistic push, chi_ph, pair rate and the first
// Method I draw, with no block-wide synchronisation.  Photons with one
// sub-step and no event are finished here; the rest are flagged and redone
// by the pair passes over the list (k_pair_count, k_pair_write).
// ---------------------------------------------------------------------------
template <class Real, int FM>
__global__ void __launch_bounds__(TILE, sizeof(Real) == 4 ? 4 : 2) k_photon_stream(PhotonArgs<Real> A) {
  const int64_t step_ = A.d_step ? *A.d_step : A.step;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real *sP = reinterpret_cast<Real *>(smem_raw);
  __shared__ long long s_meta[2];
  __shared__ BlockTally bt;
  load_tables_smem(sP, A.T.P, A.T.glp.n);
  block_tally_init(&bt);
  if (threadIdx.x == 0) s_meta[0] = *(volatile const int64_t *)A.n_active;
  __syncthreads();
  const int64_t n = s_meta[0];
  const int64_t nslots = (n + TILE - 1) / TILE * TILE;
  const Real inv_aS = sel<Real>(A.C.inv_aS, A.C.f_inv_aS);
  const Real dt = sel<Real>(A.C.dt, A.C.f_dt), wdt_max = sel<Real>(A.C.wdt_max, A.C.f_wdt_max);
  const int lane = threadIdx.x & 31;
  uint32_t batch_base = 0, batch_used = STAGE_BATCH;  // this warp's staging batch
  Tally tl;
  tl.clear();
  // nslots is a multiple of TILE: every lane of a warp runs the same iterations
  for (int64_t i = blockIdx.x * (int64_t)TILE + threadIdx.x; i < nslots;
       i += (int64_t)gridDim.x * TILE) {
    uint8_t flag = 0;
    Real x = 0, y = 0, z = 0, px = 0, py = 0, pz = 0;
    Real E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
    uint64_t pid = 0;
    if (i < n && A.ph.alive[i]) {
      x = A.ph.x[i]; y = A.ph.y[i]; z = A.ph.z[i];
      px = A.ph.px[i]; py = A.ph.py[i]; pz = A.ph.pz[i];
      get_fields<Real, FM>(A.ph, A.f, i, x, y, z, E, B);
      Real k = m_sqrt(px * px + py * py + pz * pz);
      Real chi = chi_photon(px, py, pz, E[0], E[1], E[2], B[0], B[1], B[2], inv_aS);
      Tally t0;
      t0.clear();
      RateOut<Real> ro = pair_rate(sP, A.T, A.C, chi, k, t0);
      Real wdt = ro.W * dt;
      if (wdt > wdt_max) {
        flag = 1;
        pid = A.ph.id[i];
      } else if (ro.W > (Real)0) {  // (most soft photons have W = 0: no id read)
        pid = A.ph.id[i];
        U4 r = draw(A.C, pid, step_, 0, STREAM_PAIR);
        if (wdt > unif<Real>(r.x)) flag = 1;
      }
      if (k > (Real)0) {
        Real ik = dt / k;
        x += px * ik; y += py * ik; z += pz * ik;
      }
      if (!flag) {
        tl.substeps += 1;
        tl.status |= t0.status;
        tl.domain += t0.domain;
        if (k > (Real)0) { A.ph.x[i] = x; A.ph.y[i] = y; A.ph.z[i] = z; }
      }
    }
    A.flags[i] = flag;
    // stage the flagged photons (warp-collective)
    const unsigned m = __ballot_sync(0xFFFFFFFFu, flag != 0);
    if (m) {
      const uint32_t cm = __popc(m);
      if (batch_used + cm > STAGE_BATCH) {
        uint32_t nb = 0;
        if (lane == 0) nb = atomicAdd(A.stage_n, STAGE_BATCH);
        batch_base = __shfl_sync(0xFFFFFFFFu, nb, 0);
        batch_used = 0;
      }
      if (flag) {
        const uint64_t pos = (uint64_t)batch_base + batch_used + __popc(m & ((1u << lane) - 1u));
        int32_t sidx = -1;
        if (pos < (uint64_t)A.stage_cap) {
          sidx = (int32_t)pos;
          Stage<Real> r;
          r.p[0] = px; r.p[1] = py; r.p[2] = pz;
          r.e[0] = E[0]; r.e[1] = E[1]; r.e[2] = E[2];
          r.b[0] = B[0]; r.b[1] = B[1]; r.b[2] = B[2];
          r.id_lo = (uint32_t)pid; r.id_hi = (uint32_t)(pid >> 32);
          r.w = A.ph.w[i];
          r.x[0] = x; r.x[1] = y; r.x[2] = z;
          r.slot = (uint32_t)i;
          const uint4 *src = reinterpret_cast<const uint4 *>(&r);
          uint4 *dst = reinterpret_cast<uint4 *>(A.stage + pos);
#pragma unroll
          for (int q = 0; q < (int)(sizeof(Stage<Real>) / 16); ++q) dst[q] = src[q];
          if (A.ph.tag) A.stage_tag[pos] = A.ph.tag[i];
          // the pushed position does not depend on the pair decision
          A.ph.x[i] = x; A.ph.y[i] = y; A.ph.z[i] = z;
        }
        A.stage_idx[i] = sidx;
      }
      batch_used += cm;
    }
  }
  tally_flush(&bt, tl);
  __syncthreads();
  block_tally_commit(&bt, A.o.cnt, 1);
}

// ---------------------------------------------------------------------------
// Pair passes over the list of flagged photons (list order = photon index
// order), split like the lepton emission passes: a counting pass with no
// ordering (the photon's Method I chain: at most one pair, after which the
// photon is dead), the in-place scan of the counts, and a writing pass that
// appends the e-/e+ of each pair at its scanned slot.
// ---------------------------------------------------------------------------
template <class Real> struct PhotonEntry {
  Real x, y, z, px, py, pz, k, w;
  Real E[3], B[3];
  uint64_t id;
  uint32_t tag;
  int64_t i;  // photon index
};

// List entry e >= 0: staging record e (pushed position already stored);
// e < 0: photon -e-1, which the counting pass (COUNT) pushes and stores and
// the writing pass reads back already pushed.
template <class Real, int FM, bool COUNT>
__device__ __forceinline__ void load_photon(const PhotonArgs<Real> &A, int32_t e, Real dt,
                                            PhotonEntry<Real> &P) {
  if (e >= 0) {
    Stage<Real> r;
    const uint4 *src = reinterpret_cast<const uint4 *>(A.stage + e);
    uint4 *dst = reinterpret_cast<uint4 *>(&r);
#pragma unroll
    for (int q = 0; q < (int)(sizeof(Stage<Real>) / 16); ++q) dst[q] = src[q];
    P.px = r.p[0]; P.py = r.p[1]; P.pz = r.p[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) { P.E[c] = r.e[c]; P.B[c] = r.b[c]; }
    P.id = (uint64_t)r.id_lo | ((uint64_t)r.id_hi << 32);
    P.w = r.w;
    P.x = r.x[0]; P.y = r.x[1]; P.z = r.x[2];
    P.i = r.slot;
    P.tag = A.ph.tag ? A.stage_tag[e] : 0u;
    P.k = m_sqrt(P.px * P.px + P.py * P.py + P.pz * P.pz);
    return;
  }
  const int64_t i = -(int64_t)e - 1;
  P.i = i;
  P.x = A.ph.x[i]; P.y = A.ph.y[i]; P.z = A.ph.z[i];
  P.px = A.ph.px[i]; P.py = A.ph.py[i]; P.pz = A.ph.pz[i];
  P.w = A.ph.w[i];
  P.id = A.ph.id[i];
  P.tag = A.ph.tag ? A.ph.tag[i] : 0u;
  get_fields<Real, FM>(A.ph, A.f, i, P.x, P.y, P.z, P.E, P.B);  // at the position before the push
  P.k = m_sqrt(P.px * P.px + P.py * P.py + P.pz * P.pz);
  if (COUNT && P.k > (Real)0) {
    Real ik = dt / P.k;
    P.x += P.px * ik; P.y += P.py * ik; P.z += P.pz * ik;
    A.ph.x[i] = P.x; A.ph.y[i] = P.y; A.ph.z[i] = P.z;
  }
}

// Method I for one photon (Eqs. 3, 6): 1 and the pair's (gamma_e, gamma_p,
// sub-step) on an event, else 0.
template <class Real>
__device__ __forceinline__ uint32_t pair_chain(const PhotonArgs<Real> &A, const Real *sP,
                                               const PhotonEntry<Real> &P, int64_t step_, Real dt,
                                               Tally &tl, int64_t &N, Real &ge, Real &gp,
                                               int64_t &ks) {
  const Real inv_aS = sel<Real>(A.C.inv_aS, A.C.f_inv_aS);
  const Real wdt_max = sel<Real>(A.C.wdt_max, A.C.f_wdt_max);
  Real chi = chi_photon(P.px, P.py, P.pz, P.E[0], P.E[1], P.E[2], P.B[0], P.B[1], P.B[2], inv_aS);
  RateOut<Real> ro = pair_rate(sP, A.T, A.C, chi, P.k, tl);
  N = 1;
  const Real wdt = ro.W * dt;
  if (wdt > wdt_max) {
    Real nn = m_ceil(wdt / wdt_max);
    if (nn > (Real)A.C.max_substeps) { nn = (Real)A.C.max_substeps; tl.status |= QED_STATUS_SUBSTEPS; }
    N = (int64_t)nn;
  }
  const Real dts = dt / (Real)N;
  for (int64_t s = 0; s < N; ++s) {
    U4 r = draw(A.C, P.id, step_, s, STREAM_PAIR);
    if (!(ro.W * dts > unif<Real>(r.x))) continue;
    XiOut<Real> xo = pair_xi(A.T.Yp, A.T, ro.l, unif<Real>(r.y), unif<Real>(~r.y));
    ge = xo.xi * P.k;
    gp = xo.omxi * P.k;
    if (ge < (Real)1) { ge = (Real)1; gp = P.k - (Real)1; }
    if (gp < (Real)1) { gp = (Real)1; ge = P.k - (Real)1; }
    ks = s;
    return 1u;
  }
  return 0u;
}

template <class Real, int FM>
__global__ void __launch_bounds__(TILE) k_pair_count(PhotonArgs<Real> A) {
  const int64_t step_ = A.d_step ? *A.d_step : A.step;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real *sP = reinterpret_cast<Real *>(smem_raw);
  __shared__ long long s_meta[1];
  __shared__ BlockTally bt;
  load_tables_smem(sP, A.T.P, A.T.glp.n);
  block_tally_init(&bt);
  if (threadIdx.x == 0) s_meta[0] = *(volatile const int64_t *)A.list_n;
  __syncthreads();
  const int64_t nl = s_meta[0];
  const Real dt = sel<Real>(A.C.dt, A.C.f_dt);
  const int64_t rc = A.rec_cap;
  Tally tl;
  tl.clear();
  for (int64_t h = blockIdx.x * (int64_t)TILE + threadIdx.x; h < nl; h += (int64_t)gridDim.x * TILE) {
    PhotonEntry<Real> P;
    load_photon<Real, FM, true>(A, A.list[h], dt, P);
    int64_t N = 1, ks = 0;
    Real ge = 0, gp = 0;
    const uint32_t cnt = pair_chain(A, sP, P, step_, dt, tl, N, ge, gp, ks);
    tl.substeps += N;
    tl.events += cnt;
    A.sub_cnt[h] = cnt;
    if (cnt) {
      A.ph.alive[P.i] = 0;
      if (h < rc) {
        A.rec_e[h] = ge;
        A.rec_e[rc + h] = gp;
        A.rec_k[h] = (uint32_t)ks;
      }
    }
  }
  tally_flush(&bt, tl);
  __syncthreads();
  block_tally_commit(&bt, A.o.cnt, 1);
}

template <class Real, int FM>
__global__ void __launch_bounds__(TILE) k_pair_write(PhotonArgs<Real> A) {
  const int64_t step_ = A.d_step ? *A.d_step : A.step;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real *sP = reinterpret_cast<Real *>(smem_raw);
  __shared__ long long s_meta[4];
  __shared__ BlockTally bt;
  load_tables_smem(sP, A.T.P, A.T.glp.n);  // for entries past the record capacity
  block_tally_init(&bt);
  if (threadIdx.x == 0) {
    s_meta[0] = *(volatile const int64_t *)A.list_n;
    s_meta[1] = A.sub_meta[0];  // pairs of all entries
    s_meta[2] = A.sub_meta[1];  // electron count before them
    s_meta[3] = A.sub_meta[2];  // positron count before them
  }
  __syncthreads();
  const int64_t nl = s_meta[0];
  const uint32_t total = (uint32_t)s_meta[1];
  const int64_t ne = s_meta[2], np = s_meta[3];
  const Real dt = sel<Real>(A.C.dt, A.C.f_dt);
  const int64_t rc = A.rec_cap;
  Tally tl;
  tl.clear();
  for (int64_t h = blockIdx.x * (int64_t)TILE + threadIdx.x; h < nl; h += (int64_t)gridDim.x * TILE) {
    const uint32_t off = A.sub_cnt[h];  // exclusive prefix of the counts now
    const uint32_t cnt = (h + 1 < nl ? A.sub_cnt[h + 1] : total) - off;
    if (!cnt) continue;
    PhotonEntry<Real> P;
    load_photon<Real, FM, false>(A, A.list[h], dt, P);
    Real ge = 0, gp = 0;
    int64_t ks = 0;
    if (h < rc) {
      ge = A.rec_e[h];
      gp = A.rec_e[rc + h];
      ks = A.rec_k[h];
    } else {  // past the record capacity: redo the chain (same draws, same table)
      Tally dummy;
      dummy.clear();
      int64_t N = 1;
      if (!pair_chain(A, sP, P, step_, dt, dummy, N, ge, gp, ks)) {
        tl.status |= QED_STATUS_REPLAY;  // should not happen: write a pair at rest
        ge = gp = (Real)1;
      }
    }
    const Real ik = (Real)1 / P.k;
    const Real nx = P.px * ik, ny = P.py * ik, nz = P.pz * ik;
    const U4 cid = draw(A.C, P.id, step_, ks, STREAM_PAIR_ID);
    const Real pe = m_sqrt((ge - (Real)1) * (ge + (Real)1));
    const Real pp = m_sqrt((gp - (Real)1) * (gp + (Real)1));
    if (ne + off < A.el.cap)
      write_child(A.el, ne + off, P.x, P.y, P.z, pe * nx, pe * ny, pe * nz, P.w,
                  (uint64_t)cid.x | ((uint64_t)cid.y << 32), P.E, P.B, P.tag);
    else { tl.dropped += 1; tl.status |= QED_STATUS_CAPACITY; }
    if (np + off < A.po.cap)
      write_child(A.po, np + off, P.x, P.y, P.z, pp * nx, pp * ny, pp * nz, P.w,
                  (uint64_t)cid.z | ((uint64_t)cid.w << 32), P.E, P.B, P.tag);
    else { tl.dropped += 1; tl.status |= QED_STATUS_CAPACITY; }
  }
  tally_flush(&bt, tl);
  __syncthreads();
  block_tally_commit(&bt, A.o.cnt, 1);
}

// ---------------------------------------------------------------------------
// Stable in-place compaction of dead particles (alive == 0).  Every tile loads
// its particles into registers before it publishes its count, and a tile
// writes only below the end of its own range, after every earlier tile has
// published -- so no data is overwritten before it has been read.
// ---------------------------------------------------------------------------
// Compaction tiles are COMPACT_ITEMS x 1024 particles (1024-thread CTAs, item k
// of thread i is particle k * 1024 + i of the tile, so every load and store is
// coalesced).  Tiles this large matter: a tile learns its prefix from the tile
// states of its predecessors, a warp-wide window of 32 per round trip, so the
// pass advances about 32 tiles per L2 round trip whatever the bandwidth.
constexpr int COMPACT_TILE = 1024;
template <class Real> __host__ __device__ constexpr int compact_items() { return sizeof(Real) == 4 ? 2 : 1; }

template <class Real> struct CompactArgs {
  Sp<Real> s;
  Out o;
};

template <class Real>
__global__ void __launch_bounds__(COMPACT_TILE) k_compact(CompactArgs<Real> A) {
  constexpr int CI = compact_items<Real>();
  constexpr int64_t TP = (int64_t)CI * COMPACT_TILE;  // particles per tile
  __shared__ uint32_t scan_sm[33];
  __shared__ long long s_meta[8];
  if (threadIdx.x == 0) {
    s_meta[2] = *(volatile int64_t *)A.s.d_n;
    s_meta[5] = (long long)A.o.scan.sync[2];
  }
  __syncthreads();
  const int64_t n = s_meta[2];
  const uint32_t epoch = (uint32_t)s_meta[5];
  const int64_t ntiles = (n + TP - 1) / TP;
  const bool fields = A.s.ex != nullptr;
  uint32_t status = 0;
  for (;;) {
    if (threadIdx.x == 0) s_meta[0] = (long long)atomicAdd(&A.o.scan.sync[0], 1u);
    __syncthreads();
    const int64_t t = s_meta[0];
    __syncthreads();
    if (t >= ntiles) break;
    uint32_t keep[CI];
    Real v[CI][13];
    uint64_t id[CI];
    uint32_t tg[CI];
#pragma unroll
    for (int k = 0; k < CI; ++k) {
      const int64_t i = t * TP + k * COMPACT_TILE + threadIdx.x;
      keep[k] = 0;
      id[k] = 0;
      tg[k] = 0;
      if (i < n && A.s.alive[i]) {
        keep[k] = 1;
        if (A.s.tag) tg[k] = A.s.tag[i];
        v[k][0] = A.s.x[i]; v[k][1] = A.s.y[i]; v[k][2] = A.s.z[i];
        v[k][3] = A.s.px[i]; v[k][4] = A.s.py[i]; v[k][5] = A.s.pz[i]; v[k][6] = A.s.w[i];
        id[k] = A.s.id[i];
        if (fields) {
          v[k][7] = A.s.ex[i]; v[k][8] = A.s.ey[i]; v[k][9] = A.s.ez[i];
          v[k][10] = A.s.bx[i]; v[k][11] = A.s.by[i]; v[k][12] = A.s.bz[i];
        }
      }
    }
    // destination of item k within the tile: the items of the earlier stripes,
    // then this stripe's prefix
    uint32_t excl[CI];
    uint32_t agg = 0;
#pragma unroll
    for (int k = 0; k < CI; ++k) {
      if (k > 0) __syncthreads();  // scan_sm is reused
      excl[k] = agg + block_excl_scan(keep[k], scan_sm);
      agg += scan_sm[32];
    }
    if (threadIdx.x < 32) {
      uint32_t st_tile = 0;
      uint32_t pre = lookback_warp(A.o.scan, t, epoch, agg, st_tile);
      // any lane of the walk may have given up (warp 0 runs converged here)
      const bool gave_up = __any_sync(0xFFFFFFFFu, (st_tile & QED_STATUS_TIMEOUT) != 0);
      status |= st_tile;
      if (threadIdx.x == 0) {
        s_meta[1] = pre;
        // a look-back that gave up has no valid prefix: this tile writes
        // nothing (an in-place write could land on particles an earlier tile
        // has not read yet); the result is flagged QED_STATUS_TIMEOUT
        s_meta[3] = gave_up ? 1 : 0;
        if (t == ntiles - 1 && !s_meta[3]) *A.s.d_n = (int64_t)pre + agg;
      }
    }
    __syncthreads();
    const bool skip = s_meta[3] != 0;
#pragma unroll
    for (int k = 0; k < CI; ++k) {
      if (!keep[k] || skip) continue;
      const int64_t d = s_meta[1] + excl[k];
      A.s.x[d] = v[k][0]; A.s.y[d] = v[k][1]; A.s.z[d] = v[k][2];
      A.s.px[d] = v[k][3]; A.s.py[d] = v[k][4]; A.s.pz[d] = v[k][5]; A.s.w[d] = v[k][6];
      A.s.id[d] = id[k];
      A.s.alive[d] = 1;
      if (A.s.tag) A.s.tag[d] = tg[k];
      if (fields) {
        A.s.ex[d] = v[k][7]; A.s.ey[d] = v[k][8]; A.s.ez[d] = v[k][9];
        A.s.bx[d] = v[k][10]; A.s.by[d] = v[k][11]; A.s.bz[d] = v[k][12];
      }
    }
  }
  if (threadIdx.x == 0 && status) atomicOr(&A.o.cnt->status, status);
  launch_epilogue(A.o.scan, epoch);
}

// ---------------------------------------------------------------------------
// Hole-filling compaction.  With a live particles among n, every dead slot
// below a (a hole) receives a live particle from [a, n) (a tail): the k-th
// hole in index order takes the k-th tail in index order.  Only as many
// particles move as there are holes, and every live particle below a keeps
// its index.  Count, scan, hole-list and move passes; no CTA waits on another.
// ---------------------------------------------------------------------------
constexpr int FILL_ITEMS = 8;
constexpr int FILL_CHUNK = TILE * FILL_ITEMS;
static_assert(FILL_CHUNK == CLS_CHUNK_FLAGS, "fill chunks use the class-list scratch");

template <class Real> struct FillArgs {
  Sp<Real> s;
  unsigned long long *chunk_alive;  // [chunks]
  uint32_t *chunk_off;              // [chunks][NCLS]: [0] holes before, [1] tails before
  int64_t *meta;                    // [0] n, [1] a
  int *holes;                       // hole slots in index order
};

// live flags of this thread's 8 slots of chunk c (bit j: slot first + j)
__device__ __forceinline__ uint32_t fill_bits(const uint8_t *alive, int64_t c, int64_t n,
                                              int64_t &first) {
  first = c * FILL_CHUNK + (int64_t)threadIdx.x * FILL_ITEMS;
  uint32_t bits = 0;
#pragma unroll
  for (int j = 0; j < FILL_ITEMS; ++j)
    if (first + j < n && alive[first + j]) bits |= 1u << j;
  return bits;
}

template <class Real>
__global__ void __launch_bounds__(TILE) k_fill_count(FillArgs<Real> A) {
  __shared__ uint32_t scan_sm[33];
  const int64_t n = *(volatile const int64_t *)A.s.d_n;
  const int64_t nchunks = (n + FILL_CHUNK - 1) / FILL_CHUNK;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    int64_t first;
    const uint32_t bits = fill_bits(A.s.alive, c, n, first);
    block_excl_scan(__popc(bits), scan_sm);
    if (threadIdx.x == 0) A.chunk_alive[c] = scan_sm[32];
    __syncthreads();
  }
}

// One CTA: a, the boundary chunk's split, and each chunk's hole and tail offsets.
__global__ void __launch_bounds__(CLS_SCAN_THREADS) k_fill_scan(const uint8_t *alive,
                                                                 int64_t *d_n,
                                                                 FillArgs<float> A) {
  __shared__ unsigned long long tot;
  __shared__ unsigned long long sm[33];
  __shared__ uint32_t xs;
  const int64_t n = *(volatile const int64_t *)d_n;
  const int64_t nchunks = (n + FILL_CHUNK - 1) / FILL_CHUNK;
  if (threadIdx.x == 0) { tot = 0; xs = 0; }
  __syncthreads();
  unsigned long long mine = 0;
  for (int64_t c = threadIdx.x; c < nchunks; c += blockDim.x) mine += A.chunk_alive[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xFFFFFFFFu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&tot, mine);
  __syncthreads();
  const int64_t a = (int64_t)tot;
  // live particles of the boundary chunk below a
  const int64_t cb = a / FILL_CHUNK, b0 = cb * FILL_CHUNK;
  uint32_t xl = 0;
  for (int64_t i = b0 + threadIdx.x; i < a; i += blockDim.x) xl += alive[i] ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) xl += __shfl_xor_sync(0xFFFFFFFFu, xl, o);
  if ((threadIdx.x & 31) == 0 && xl) atomicAdd(&xs, xl);
  __syncthreads();
  const uint32_t x = xs;
  if (threadIdx.x == 0) {
    A.meta[0] = n;
    A.meta[1] = a;
    *d_n = a;
  }
  int64_t carry_h = 0, carry_t = 0;
  const int64_t per_round = (int64_t)blockDim.x * CLS_SCAN_PER_THREAD;
  for (int64_t r0 = 0; r0 < nchunks; r0 += per_round) {
    const int64_t c0 = r0 + (int64_t)threadIdx.x * CLS_SCAN_PER_THREAD;
    uint32_t hv[CLS_SCAN_PER_THREAD], tv[CLS_SCAN_PER_THREAD];
    uint32_t hs = 0, ts = 0;
#pragma unroll
    for (int j = 0; j < CLS_SCAN_PER_THREAD; ++j) {
      const int64_t c = c0 + j;
      hv[j] = tv[j] = 0;
      if (c < nchunks) {
        const int64_t lo = c * FILL_CHUNK, hi = lo + FILL_CHUNK < n ? lo + FILL_CHUNK : n;
        const uint32_t al = (uint32_t)A.chunk_alive[c];
        if (hi <= a) {
          hv[j] = (uint32_t)(hi - lo) - al;
        } else if (lo >= a) {
          tv[j] = al;
        } else {
          hv[j] = (uint32_t)(a - lo) - x;
          tv[j] = al - x;
        }
      }
      hs += hv[j];
      ts += tv[j];
    }
    const unsigned long long v = (unsigned long long)hs | ((unsigned long long)ts << 32);
    const unsigned long long e = block_excl_scan64(v, sm), tt = sm[32];
    uint32_t rh = (uint32_t)e, rt = (uint32_t)(e >> 32);
#pragma unroll
    for (int j = 0; j < CLS_SCAN_PER_THREAD; ++j) {
      const int64_t c = c0 + j;
      if (c < nchunks) {
        A.chunk_off[c * NCLS + 0] = (uint32_t)(carry_h + rh);
        A.chunk_off[c * NCLS + 1] = (uint32_t)(carry_t + rt);
      }
      rh += hv[j];
      rt += tv[j];
    }
    carry_h += (int64_t)(uint32_t)tt;
    carry_t += (int64_t)(uint32_t)(tt >> 32);
  }
}

template <class Real>
__global__ void __launch_bounds__(TILE) k_fill_holes(FillArgs<Real> A) {
  __shared__ uint32_t scan_sm[33];
  const int64_t n = A.meta[0], a = A.meta[1];
  const int64_t nchunks = (a + FILL_CHUNK - 1) / FILL_CHUNK;  // chunks with slots below a
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    int64_t first;
    uint32_t bits = fill_bits(A.s.alive, c, n, first);
    uint32_t hole = 0;
#pragma unroll
    for (int j = 0; j < FILL_ITEMS; ++j)
      if (first + j < a && !(bits & (1u << j))) hole |= 1u << j;
    uint32_t k = A.chunk_off[c * NCLS + 0] + block_excl_scan(__popc(hole), scan_sm);
    __syncthreads();
    while (hole) {
      const int j = __ffs(hole) - 1;
      hole &= hole - 1;
      A.holes[k++] = (int)(first + j);
    }
  }
}

template <class Real>
__global__ void __launch_bounds__(TILE) k_fill_move(FillArgs<Real> A) {
  __shared__ uint32_t scan_sm[33];
  const int64_t n = A.meta[0], a = A.meta[1];
  const int64_t c_lo = a / FILL_CHUNK, nchunks = (n + FILL_CHUNK - 1) / FILL_CHUNK;
  const Sp<Real> &S = A.s;
  const bool fields = S.ex != nullptr;
  for (int64_t c = c_lo + blockIdx.x; c < nchunks; c += gridDim.x) {
    int64_t first;
    const uint32_t bits = fill_bits(S.alive, c, n, first);
    uint32_t tail = 0;
#pragma unroll
    for (int j = 0; j < FILL_ITEMS; ++j)
      if (first + j >= a && (bits & (1u << j))) tail |= 1u << j;
    uint32_t k = A.chunk_off[c * NCLS + 1] + block_excl_scan(__popc(tail), scan_sm);
    __syncthreads();
    while (tail) {
      const int j = __ffs(tail) - 1;
      tail &= tail - 1;
      const int64_t i = first + j, d = A.holes[k++];
      S.x[d] = S.x[i]; S.y[d] = S.y[i]; S.z[d] = S.z[i];
      S.px[d] = S.px[i]; S.py[d] = S.py[i]; S.pz[d] = S.pz[i];
      S.w[d] = S.w[i];
      S.id[d] = S.id[i];
      if (S.tag) S.tag[d] = S.tag[i];
      if (fields) {
        S.ex[d] = S.ex[i]; S.ey[d] = S.ey[i]; S.ez[d] = S.ez[i];
        S.bx[d] = S.bx[i]; S.by[d] = S.by[i]; S.bz[d] = S.bz[i];
      }
      S.alive[d] = 1;
    }
  }
}

// ---------------------------------------------------------------------------
// Number of live particles (alive != 0) among the first *d_n, added to *out.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TILE) k_count_alive(const uint8_t *alive, const int64_t *d_n,
                                                      unsigned long long *out) {
  const int64_t n = *(volatile const int64_t *)d_n;
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)TILE + threadIdx.x; i < n; i += (int64_t)gridDim.x * TILE)
    c += alive[i] ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ---------------------------------------------------------------------------
// Snapshot of the photon count at the start of a fused step.
// ---------------------------------------------------------------------------
__global__ void k_snapshot(const int64_t *src, int64_t *dst) { *dst = *src; }

// ---------------------------------------------------------------------------
// Isolated sampler (xi at given chi, gamma; r2 from Philox(i, step)).
// ---------------------------------------------------------------------------
struct SampleArgs {
  const float *chi, *gamma;
  float *xi;
  int64_t n, step;
  Consts C;
  Tables<float> T;
  Out o;
  const uint32_t *mlp_frag;
  const float *mlp_w;
  int use_mlp;
  int emit_lanes, scan_draws;  // chain scheduling (QED_SCHED_EMIT_LANES, _SCAN_DRAWS)
};

__global__ void __launch_bounds__(TILE) k_sample_xi(SampleArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *sR = reinterpret_cast<float *>(smem_raw);
  float *sF = sR + A.T.gl.n;
  uint32_t *s_frag = reinterpret_cast<uint32_t *>(
      smem_raw + (((size_t)A.T.gl.n * (1 + A.T.gy.n) * sizeof(float) + 15) & ~(size_t)15));
  float *s_fw = reinterpret_cast<float *>(s_frag + MLP_FRAG_WORDS);
  load_tables_smem(sR, A.T.R, A.T.gl.n);
  load_tables_smem(sF, A.T.F, A.T.gl.n * A.T.gy.n);
  if (A.use_mlp) mlp_stage(s_frag, s_fw, A.mlp_frag, A.mlp_w);
  __syncthreads();
  Tally tl;
  tl.clear();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform loop (the learned sampler is a warp-collective call)
  for (int64_t ib = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); ib < A.n; ib += stride) {
    const int64_t i = ib + (threadIdx.x & 31);
    const bool active = i < A.n;
    float chi = active ? __ldcs(A.chi + i) : 1.f, g = active ? __ldcs(A.gamma + i) : 1e3f;
    RateOut<float> ro = photon_rate(sR, sF, A.T, A.C, chi, g, tl);
    U4 r = draw(A.C, (uint64_t)i, A.step, 0, STREAM_EMIT);
    const float kap = photon_kappa(ro.kmin, unif<float>(r.y), unif<float>(~r.y));
    float Y = 0.f;
    bool in_mlp = false;
    if (A.use_mlp) {
      const float lchi = logf(chi);
      in_mlp = lchi >= MLP_L_LO && lchi <= MLP_L_HI && kap >= MLP_K_LO && kap <= MLP_K_HI;
      Y = mlp_infer_warp(s_frag, s_fw, (lchi - MLP_LC) / MLP_LS, (kap - MLP_KC) / MLP_KS) +
          mlp_baseline(kap);
    }
    if (!active) continue;
    float xi = 0.f;
    if (ro.W > 0.f) {
      if (!in_mlp) Y = photon_lndelta_table(A.T.Y, A.T, ro.l, kap, tl);
      xi = xi_from_lndelta(chi, Y).xi;
    }
    __stcs(A.xi + i, xi);
  }
  if (tl.status) atomicOr(&A.o.cnt->status, tl.status);
}

// ---------------------------------------------------------------------------
// Parity helpers: rates and inverse CDF at given inputs (tables in global).
// ---------------------------------------------------------------------------
template <class Real> struct EvalArgs {
  int which;
  const double *chi, *gamma;
  const uint32_t *word;
  double *out;
  int64_t n;
  Consts C;
  Tables<Real> T;
};

template <class Real> __global__ void k_eval_rates(EvalArgs<Real> A) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  Tally tl;
  tl.clear();
  Real chi = (Real)A.chi[i], g = (Real)A.gamma[i];
  if (A.which == 0)
    A.out[i] = (double)photon_rate(A.T.R, A.T.F, A.T, A.C, chi, g, tl).W;
  else
    A.out[i] = (double)pair_rate(A.T.P, A.T, A.C, chi, g, tl).W;
}

template <class Real> __global__ void k_eval_xi(EvalArgs<Real> A) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  Tally tl;
  tl.clear();
  Real chi = (Real)A.chi[i];
  uint32_t w = A.word[i];
  if (A.which == 0) {
    Real g = (Real)A.gamma[i];
    RateOut<Real> ro = photon_rate(A.T.R, A.T.F, A.T, A.C, chi, g, tl);
    XiOut<Real> xo = photon_xi(A.T.Y, A.T, ro.l, chi, ro.kmin, unif<Real>(w), unif<Real>(~w), tl);
    A.out[i] = (double)xo.xi;
  } else {
    RateOut<Real> ro = pair_rate(A.T.P, A.T, A.C, chi, (Real)1e6, tl);
    Real l = ro.l;
    if (!(chi >= sel<Real>(A.C.chi_pair_min, A.C.f_chi_pair_min))) l = A.T.glp.lo;
    XiOut<Real> xo = pair_xi(A.T.Yp, A.T, l, unif<Real>(w), unif<Real>(~w));
    A.out[i] = (double)xo.xi;
  }
}

// chi of every particle of a species from its momentum and per-particle
// fields (Eq. 2 for leptons, Eq. 3 for photons), in the context's precision,
// by the same functions the step kernels use (parity hook).
template <class Real> __global__ void k_eval_chi(Sp<Real> S, Real inv_aS, double *out) {
  const int64_t n = *(volatile const int64_t *)S.d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Real px = S.px[i], py = S.py[i], pz = S.pz[i];
    Real chi;
    if (S.q == (Real)0) {
      chi = chi_photon(px, py, pz, S.ex[i], S.ey[i], S.ez[i], S.bx[i], S.by[i], S.bz[i], inv_aS);
    } else {
      const Real g = m_sqrt((Real)1 + px * px + py * py + pz * pz);
      chi = chi_lepton(px, py, pz, g, S.ex[i], S.ey[i], S.ez[i], S.bx[i], S.by[i], S.bz[i], inv_aS);
    }
    out[i] = (double)chi;
  }
}

// Learned inverse CDF at given inputs (parity and spectral-error hook): xi
// of the photon sampler at (chi, gamma) for the uniform word w, through the
// network where (ln chi, kappa) lies in its domain, else through the inverse
// table -- exactly the choice the step kernels make.  Warp-uniform loop (the
// network is a warp-collective call); rates from the global-memory tables.
__global__ void __launch_bounds__(TILE) k_eval_xi_mlp(EvalArgs<float> A, const uint32_t *frag,
                                                      const float *w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *s_frag = reinterpret_cast<uint32_t *>(smem_raw);
  float *s_fw = reinterpret_cast<float *>(s_frag + MLP_FRAG_WORDS);
  mlp_stage(s_frag, s_fw, frag, w);
  __syncthreads();
  Tally tl;
  tl.clear();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t ib = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); ib < A.n; ib += stride) {
    const int64_t i = ib + (threadIdx.x & 31);
    const bool active = i < A.n;
    const float chi = active ? (float)A.chi[i] : 1.f, g = active ? (float)A.gamma[i] : 1e3f;
    const uint32_t wd = active ? A.word[i] : 0u;
    RateOut<float> ro = photon_rate(A.T.R, A.T.F, A.T, A.C, chi, g, tl);
    const float kap = photon_kappa(ro.kmin, unif<float>(wd), unif<float>(~wd));
    const float lchi = logf(chi);
    const bool in_mlp = lchi >= MLP_L_LO && lchi <= MLP_L_HI && kap >= MLP_K_LO && kap <= MLP_K_HI;
    float Y = mlp_infer_warp(s_frag, s_fw, (lchi - MLP_LC) / MLP_LS, (kap - MLP_KC) / MLP_KS) +
              mlp_baseline(kap);
    if (!active) continue;
    double xi = 0.0;
    if (ro.W > 0.f) {
      if (!in_mlp) Y = photon_lndelta_table(A.T.Y, A.T, ro.l, kap, tl);
      xi = (double)xi_from_lndelta(chi, Y).xi;
    }
    A.out[i] = xi;
  }
}

// ---------------------------------------------------------------------------
// Standing wave E = 2 a0 cos x (0, cos t, sin t), B = 2 a0 sin x (0, cos t,
// sin t) on grid[nz][ny][nx][8].  Each block computes the nx node values of
// one x-row once (FP64 cos/sin) and streams them over its (y, z) rows.
// ---------------------------------------------------------------------------
__global__ void k_fill_standing_wave(float *grid, int nx, int ny, int nz, double x0, double dx,
                                     double a0, double t) {
  extern __shared__ __align__(16) float4 srow[];  // [nx][2]
  const double ct = cos(t), st = sin(t);
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    double x = x0 + (double)i * dx;
    double cx = 2.0 * a0 * cos(x), sx = 2.0 * a0 * sin(x);
    srow[2 * i] = make_float4(0.f, (float)(cx * ct), (float)(cx * st), 0.f);
    srow[2 * i + 1] = make_float4((float)(sx * ct), (float)(sx * st), 0.f, 0.f);
  }
  __syncthreads();
  const int64_t rows = (int64_t)ny * nz;
  const int64_t total = rows * nx * 2;  // float4 units
  float4 *g4 = reinterpret_cast<float4 *>(grid);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t within = q % (2 * (int64_t)nx);
    __stcs(g4 + q, srow[within]);
  }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers
// ---------------------------------------------------------------------------
Consts consts_of(const qed_ctx *c) {
  Consts k{};
  k.a_S = c->cfg.a_S;
  k.alpha = c->cfg.alpha;
  k.dt = c->cfg.dt;
  k.wdt_max = c->cfg.wdt_max;
  k.xi_min_energy = c->cfg.xi_min_energy;
  k.generator = c->cfg.generator;
  k.chi_pair_min = c->cfg.chi_pair_min;
  k.spec_lo = c->cfg.spec_lo;
  k.spec_scale = 64.0 / log(c->cfg.spec_hi / c->cfg.spec_lo);
  k.seed = c->cfg.seed;
  k.max_substeps = c->cfg.max_substeps;
  k.pair_sign = c->cfg.pair_sign;
  k.inv_aS = 1.0 / c->cfg.a_S;
  k.alpha_aS = c->cfg.alpha * c->cfg.a_S;
  k.f_dt = (float)k.dt;
  k.f_wdt_max = (float)k.wdt_max;
  k.f_xi_min_energy = (float)k.xi_min_energy;
  k.f_chi_pair_min = (float)k.chi_pair_min;
  k.f_spec_lo = (float)k.spec_lo;
  k.f_spec_scale = (float)k.spec_scale;
  k.f_inv_aS = (float)k.inv_aS;
  k.f_alpha_aS = (float)k.alpha_aS;
  for (int r = 0; r < 10; ++r) {
    k.rk[2 * r] = (uint32_t)k.seed + (uint32_t)r * 0x9E3779B9u;
    k.rk[2 * r + 1] = (uint32_t)(k.seed >> 32) + (uint32_t)r * 0xBB67AE85u;
  }
  return k;
}

Out out_of(const qed_ctx *c) {
  return Out{c->d_counters, ScanState{c->tile_state, c->sync, c->max_tiles}};
}

template <class Real> size_t lepton_smem(const qed_ctx *c) {
  return sizeof(Real) * ((size_t)c->gl.n + (size_t)c->gl.n * c->gy.n);
}

static cudaError_t launch_flag_list(qed_ctx *c, const uint8_t *flags, uint8_t want, const int64_t *n0,
                                    const int64_t *n1, const Out &o, const int32_t *stage_idx,
                                    cudaStream_t st) {
  HeavyListArgs h{};
  h.flags = flags;
  h.want = want;
  h.stage_idx = stage_idx;
  h.list = c->heavy_list;
  h.count = c->heavy_n;
  h.n0 = n0;
  h.n1 = n1;
  h.o = o;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heavy_list, TILE, 0);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_ORDER);
  k_heavy_list<<<c->num_sms * per_sm, TILE, 0, st>>>(h);
  c->launches += 1;
  return cudaGetLastError();
}

template <class Real, int FM>
static cudaError_t launch_push(qed_ctx *c, const LeptonArgs<Real> &a, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lepton_push<Real, FM>, TILE, 0);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_STREAM);
  k_lepton_push<Real, FM><<<c->num_sms * per_sm, TILE, 0, st>>>(a);
  c->launches += 1;
  return cudaGetLastError();
}

// A persistent launch of an emission kernel that stages the FP32 rate and
// forward tables (and, when `mlp` is set, the learned sampler) in shared memory.
template <class Real, class Kern>
static cudaError_t launch_tables_kernel(qed_ctx *c, Kern kern, const LeptonArgs<Real> &a, bool mlp,
                                        int group, cudaStream_t st, size_t extra = 0) {
  size_t sm = sizeof(Real) == 8 ? 0 : lepton_smem<Real>(c);
  if (sm && mlp) sm = ((sm + 15) & ~(size_t)15) + MLP_SMEM_BYTES;
  if (extra) sm = ((sm + 15) & ~(size_t)15) + extra;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TILE, sm);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, group);
  kern<<<c->num_sms * per_sm, TILE, sm, st>>>(a);
  c->launches += 1;
  return cudaGetLastError();
}

// A persistent launch of a kernel without dynamic shared memory.
template <class Real, class Kern>
static cudaError_t launch_plain_kernel(qed_ctx *c, Kern kern, const LeptonArgs<Real> &a,
                                       cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TILE, 0);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_ORDER);
  kern<<<c->num_sms * per_sm, TILE, 0, st>>>(a);
  c->launches += 1;
  return cudaGetLastError();
}

// The class list of the streaming pass's flags (three launches).
static cudaError_t launch_class_lists(qed_ctx *c, const int64_t *n0, const int64_t *n1,
                                      cudaStream_t st) {
  ClassListArgs a{};
  a.flags = c->heavy_flags;
  a.n0 = n0;
  a.n1 = n1;
  a.list = c->heavy_list;
  a.chunk_cnt = c->cls_chunk_cnt;
  a.chunk_off = c->cls_chunk_off;
  a.off = c->cls_off;
  a.stage_idx = c->stage_idx;
  a.stage_n = c->stage_n;
  a.cnt = c->d_counters;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cls_count, TILE, 0);
  if (e != cudaSuccess) return e;
  const int grid = c->num_sms * (per_sm > 0 ? per_sm : 1);
  k_cls_count<<<grid, TILE, 0, st>>>(a);
  k_cls_scan<<<1, CLS_SCAN_THREADS, 0, st>>>(a);
  k_cls_scatter<<<grid, TILE, 0, st>>>(a);
  c->launches += 3;
  return cudaGetLastError();
}

static cudaError_t launch_sub_scan(qed_ctx *c, const int64_t *n_entries, int64_t *out1_n,
                                   int64_t out1_cap, int64_t *out2_n, int64_t out2_cap,
                                   cudaStream_t st) {
  SubScanArgs a{};
  a.cnt = c->sub_cnt;
  a.replay_n = c->replay_n;
  a.n_entries = n_entries;
  a.sub_meta = c->sub_meta;
  a.out1_n = out1_n;
  a.out1_cap = out1_cap;
  a.out2_n = out2_n;
  a.out2_cap = out2_cap;
  a.o = out_of(c);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sub_scan, TILE, 0);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_ORDER);
  k_sub_scan<<<c->num_sms * per_sm, TILE, 0, st>>>(a);
  c->launches += 1;
  return cudaGetLastError();
}

// Emission: the streaming pass finishes the particles that surely have one
// sub-step and no event and classes the rest; the class list orders them
// (class 1 first, each class in particle order); the counting pass, the scan
// and the writing pass append their photons in that order.
template <class Real, int FM, int MODE>
static cudaError_t launch_lepton_t(qed_ctx *c, const LeptonArgs<Real> &a, cudaStream_t st) {
  if (MODE == MODE_PUSH) return launch_push<Real, FM>(c, a, st);
  cudaError_t e = launch_tables_kernel<Real>(c, k_lepton_stream<Real, FM, MODE>, a, false,
                                             QED_TUNE_STREAM, st, stream_prefetch_bytes<Real, FM>());
  if (e == cudaSuccess) e = prof_mark(c, 1, st);
  if (e == cudaSuccess) e = launch_class_lists(c, a.sp[0].d_n, a.nsp > 1 ? a.sp[1].d_n : nullptr, st);
  if (e == cudaSuccess) e = prof_mark(c, 2, st);
  if (e == cudaSuccess)
    e = a.use_mlp && sizeof(Real) == 4
            ? launch_tables_kernel<Real>(c, k_substep_count<Real, FM, MODE, true>, a, true,
                                         QED_TUNE_CHAINS, st)
            : launch_tables_kernel<Real>(c, k_substep_count<Real, FM, MODE, false>, a, false,
                                         QED_TUNE_CHAINS, st);
  if (e == cudaSuccess) e = prof_mark(c, 3, st);
  if (e == cudaSuccess) e = launch_sub_scan(c, c->cls_off + NCLS, a.ph.d_n, a.ph.cap, nullptr, 0, st);
  if (e == cudaSuccess) e = prof_mark(c, 4, st);
  if (e == cudaSuccess) e = launch_plain_kernel<Real>(c, k_substep_write_coop<Real, FM, MODE>, a, st);
  if (e == cudaSuccess)
    e = launch_tables_kernel<Real>(c, k_substep_replay<Real, FM, MODE>, a, false, QED_TUNE_CHAINS, st);
  if (e == cudaSuccess) e = prof_mark(c, 5, st);
  return e;
}

template <class Real, int MODE>
static cudaError_t launch_lepton_m(qed_ctx *c, const LeptonArgs<Real> &a, int fm, cudaStream_t st) {
  if (fm == QED_FIELDS_UNIFORM) return launch_lepton_t<Real, FM_UNIFORM, MODE>(c, a, st);
  if (fm == QED_FIELDS_PER_PARTICLE) return launch_lepton_t<Real, FM_PER_PARTICLE, MODE>(c, a, st);
  return launch_lepton_t<Real, FM_GRID, MODE>(c, a, st);
}

cudaError_t launch_lepton_onepass(qed_ctx *c, const qed_species *s0, const qed_species *s1,
                                  const qed_species *ph, const qed_fields *f, int64_t step,
                                  int mode, cudaStream_t st);

template <class Real>
cudaError_t launch_lepton(qed_ctx *c, const qed_species *s0, const qed_species *s1,
                          const qed_species *ph, const qed_fields *f, int64_t step, int mode,
                          cudaStream_t st) {
  if (sizeof(Real) == 4 && mode != MODE_PUSH && c->cfg.append_order == QED_APPEND_ANY &&
      c->cfg.generator == QED_GEN_METHOD_I) {
    // marks: 1 after the single-pass kernel (recorded by it), 2..5 after the
    // learned sampler's dense pass, if any
    cudaError_t e = launch_lepton_onepass(c, s0, s1, ph, f, step, mode, st);
    for (int k = 2; k <= 5 && e == cudaSuccess; ++k) e = prof_mark(c, k, st);
    return e;
  }
  LeptonArgs<Real> a{};
  a.sp[0] = to_sp<Real>(s0);
  a.nsp = s1 ? 2 : 1;
  if (s1) a.sp[1] = to_sp<Real>(s1);
  a.ph = to_sp<Real>(ph);
  a.f = to_fld<Real>(f);
  a.C = consts_of(c);
  a.T = tables_of<Real>(c);
  a.o = out_of(c);
  a.step = step;
  a.heavy_flags = c->heavy_flags;
  a.heavy_list = c->heavy_list;
  a.heavy_n = c->heavy_n;
  a.cls_off = c->cls_off;
  a.sub_cnt = c->sub_cnt;
  a.sub_gf = static_cast<Real *>(c->sub_gf);
  a.rec_e = static_cast<Real *>(c->rec_e);
  a.rec_k = c->rec_k;
  a.rec_cap = c->rec_cap;
  a.stage = static_cast<Stage<Real> *>(c->stage);
  a.stage_tag = c->stage_tag;
  a.stage_idx = c->stage_idx;
  a.stage_n = c->stage_n;
  a.stage_cap = c->stage_cap;
  a.sub_meta = c->sub_meta;
  a.replay_list = c->stage_idx;  // free once the class list is built
  a.replay_n = c->replay_n;
  a.mlp_frag = c->mlp_frag;
  a.mlp_w = c->mlp_w;
  a.use_mlp = c->cfg.sampler == QED_SAMPLER_MLP && c->mlp_ready;
  a.emit_lanes = sched_param(c, QED_SCHED_EMIT_LANES);
  a.scan_draws = sched_param(c, QED_SCHED_SCAN_DRAWS);
  a.d_step = c->use_dstep ? c->d_step : nullptr;
  if (mode == MODE_PUSH) return launch_lepton_m<Real, MODE_PUSH>(c, a, f->mode, st);
  if (mode == MODE_EMIT) return launch_lepton_m<Real, MODE_EMIT>(c, a, f->mode, st);
  return launch_lepton_m<Real, MODE_FUSED>(c, a, f->mode, st);
}

template <class Real, int FM>
static cudaError_t launch_photon_t(qed_ctx *c, const PhotonArgs<Real> &a, cudaStream_t st) {
  size_t sm = sizeof(Real) * (size_t)c->glp.n;
  int per_sm = 0;
  cudaError_t e = cudaMemsetAsync(a.stage_n, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_photon_stream<Real, FM>, TILE, sm);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_PHOTON);
  k_photon_stream<Real, FM><<<c->num_sms * per_sm, TILE, sm, st>>>(a);
  c->launches += 1;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = prof_mark(c, 6, st);
  if (e == cudaSuccess) e = launch_flag_list(c, a.flags, 1, a.n_active, nullptr, a.o, a.stage_idx, st);
  if (e != cudaSuccess) return e;
  // pairs: counting pass, scan (advances both lepton counts), writing pass
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_count<Real, FM>, TILE, sm);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_PHOTON);
  k_pair_count<Real, FM><<<c->num_sms * per_sm, TILE, sm, st>>>(a);
  c->launches += 1;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_sub_scan(c, a.list_n, a.el.d_n, a.el.cap, a.po.d_n, a.po.cap, st);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_write<Real, FM>, TILE, sm);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_PHOTON);
  k_pair_write<Real, FM><<<c->num_sms * per_sm, TILE, sm, st>>>(a);
  c->launches += 1;
  return cudaGetLastError();
}

template <class Real>
cudaError_t launch_photon(qed_ctx *c, const qed_species *g, const qed_species *e,
                          const qed_species *p, const int64_t *n_active, const qed_fields *f,
                          int64_t step, cudaStream_t st) {
  PhotonArgs<Real> a{};
  a.ph = to_sp<Real>(g);
  a.el = to_sp<Real>(e);
  a.po = to_sp<Real>(p);
  a.n_active = n_active;
  a.f = to_fld<Real>(f);
  a.C = consts_of(c);
  a.T = tables_of<Real>(c);
  a.o = out_of(c);
  a.step = step;
  a.flags = c->heavy_flags;
  a.list = c->heavy_list;
  a.list_n = c->heavy_n;
  a.stage = static_cast<Stage<Real> *>(c->stage);
  a.stage_tag = c->stage_tag;
  a.stage_idx = c->stage_idx;
  a.stage_n = c->stage_n;
  a.stage_cap = c->stage_cap;
  a.sub_cnt = c->sub_cnt;
  a.sub_meta = c->sub_meta;
  a.rec_e = static_cast<Real *>(c->rec_e);
  a.rec_k = c->rec_k;
  a.rec_cap = c->rec_cap;
  a.d_step = c->use_dstep ? c->d_step : nullptr;
  if (f->mode == QED_FIELDS_UNIFORM) return launch_photon_t<Real, FM_UNIFORM>(c, a, st);
  if (f->mode == QED_FIELDS_PER_PARTICLE) return launch_photon_t<Real, FM_PER_PARTICLE>(c, a, st);
  return launch_photon_t<Real, FM_GRID>(c, a, st);
}

template <class Real>
cudaError_t launch_compact(qed_ctx *c, const qed_species *s, cudaStream_t st) {
  CompactArgs<Real> a{};
  a.s = to_sp<Real>(s);
  a.o = out_of(c);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_compact<Real>, COMPACT_TILE, 0);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_COMPACT);
  k_compact<Real><<<c->num_sms * per_sm, COMPACT_TILE, 0, st>>>(a);
  c->launches += 1;
  return cudaGetLastError();
}

template <class Real>
cudaError_t launch_compact_fill(qed_ctx *c, const qed_species *s, cudaStream_t st) {
  FillArgs<Real> a{};
  a.s = to_sp<Real>(s);
  a.chunk_alive = c->cls_chunk_cnt;
  a.chunk_off = c->cls_chunk_off;
  a.meta = c->fill_meta;
  a.holes = c->heavy_list;
  FillArgs<float> af{};  // the scan reads only the shared scratch
  af.chunk_alive = a.chunk_alive;
  af.chunk_off = a.chunk_off;
  af.meta = a.meta;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fill_count<Real>, TILE, 0);
  if (e != cudaSuccess) return e;
  const int grid = c->num_sms * (per_sm > 0 ? per_sm : 1);
  k_fill_count<Real><<<grid, TILE, 0, st>>>(a);
  k_fill_scan<<<1, CLS_SCAN_THREADS, 0, st>>>(s->alive, s->d_n, af);
  k_fill_holes<Real><<<grid, TILE, 0, st>>>(a);
  k_fill_move<Real><<<grid, TILE, 0, st>>>(a);
  c->launches += 4;
  return cudaGetLastError();
}

cudaError_t launch_count_alive(qed_ctx *c, const qed_species *s, int64_t *out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t), st);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_alive, TILE, 0);
  if (e != cudaSuccess) return e;
  k_count_alive<<<c->num_sms * (per_sm > 0 ? per_sm : 1), TILE, 0, st>>>(
      s->alive, s->d_n, reinterpret_cast<unsigned long long *>(out));
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_snapshot(qed_ctx *c, const int64_t *src, int64_t *dst, cudaStream_t st) {
  k_snapshot<<<1, 1, 0, st>>>(src, dst);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_sample_xi(qed_ctx *c, const float *chi, const float *gamma, float *xi,
                             int64_t n, int64_t step, cudaStream_t st) {
  SampleArgs a{};
  a.chi = chi; a.gamma = gamma; a.xi = xi; a.n = n; a.step = step;
  a.C = consts_of(c);
  a.T = tables_of<float>(c);
  a.o = out_of(c);
  a.mlp_frag = c->mlp_frag;
  a.mlp_w = c->mlp_w;
  a.use_mlp = c->cfg.sampler == QED_SAMPLER_MLP && c->mlp_ready;
  size_t sm = lepton_smem<float>(c);
  if (a.use_mlp) sm = ((sm + 15) & ~(size_t)15) + MLP_SMEM_BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_sample_xi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample_xi, TILE, sm);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_COMPACT);
  k_sample_xi<<<c->num_sms * per_sm, TILE, sm, st>>>(a);
  c->launches += 1;
  return cudaGetLastError();
}

template <class Real>
cudaError_t launch_eval(qed_ctx *c, int kind, int which, const double *chi, const double *gamma,
                        const uint32_t *word, double *out, int64_t n, cudaStream_t st) {
  EvalArgs<Real> a{};
  a.which = which; a.chi = chi; a.gamma = gamma; a.word = word; a.out = out; a.n = n;
  a.C = consts_of(c);
  a.T = tables_of<Real>(c);
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (blocks == 0) return cudaSuccess;
  if (kind == 0) k_eval_rates<Real><<<blocks, 256, 0, st>>>(a);
  else k_eval_xi<Real><<<blocks, 256, 0, st>>>(a);
  c->launches += 1;
  return cudaGetLastError();
}

template <class Real> cudaError_t launch_eval_chi(qed_ctx *c, const qed_species *s, double *out,
                                                   cudaStream_t st) {
  const Consts C = consts_of(c);
  k_eval_chi<Real><<<c->num_sms * 4, 256, 0, st>>>(to_sp<Real>(s), sizeof(Real) == 8 ? (Real)C.inv_aS : (Real)C.f_inv_aS,
                                                   out);
  c->launches += 1;
  return cudaGetLastError();
}
template cudaError_t launch_eval_chi<float>(qed_ctx *, const qed_species *, double *, cudaStream_t);
template cudaError_t launch_eval_chi<double>(qed_ctx *, const qed_species *, double *, cudaStream_t);

cudaError_t launch_eval_xi_mlp(qed_ctx *c, const double *chi, const double *gamma,
                               const uint32_t *word, double *out, int64_t n, cudaStream_t st) {
  EvalArgs<float> a{};
  a.which = 0; a.chi = chi; a.gamma = gamma; a.word = word; a.out = out; a.n = n;
  a.C = consts_of(c);
  a.T = tables_of<float>(c);
  if (n == 0) return cudaSuccess;
  const size_t sm = MLP_SMEM_BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_eval_xi_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int64_t blocks = (n + TILE - 1) / TILE;
  if (blocks > (int64_t)c->num_sms * 8) blocks = (int64_t)c->num_sms * 8;
  k_eval_xi_mlp<<<(unsigned)blocks, TILE, sm, st>>>(a, c->mlp_frag, c->mlp_w);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_fill(qed_ctx *c, float *grid, int nx, int ny, int nz, double x0, double dx,
                        double a0, double t, cudaStream_t st) {
  size_t sm = sizeof(float4) * 2 * (size_t)nx;
  cudaError_t e = cudaFuncSetAttribute(k_fill_standing_wave,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_fill_standing_wave<<<c->num_sms * 4, 256, sm, st>>>(grid, nx, ny, nz, x0, dx, a0, t);
  c->launches += 1;
  return cudaGetLastError();
}

template cudaError_t launch_lepton<float>(qed_ctx *, const qed_species *, const qed_species *,
                                          const qed_species *, const qed_fields *, int64_t, int,
                                          cudaStream_t);
template cudaError_t launch_lepton<double>(qed_ctx *, const qed_species *, const qed_species *,
                                           const qed_species *, const qed_fields *, int64_t, int,
                                           cudaStream_t);
template cudaError_t launch_photon<float>(qed_ctx *, const qed_species *, const qed_species *,
                                          const qed_species *, const int64_t *, const qed_fields *,
                                          int64_t, cudaStream_t);
template cudaError_t launch_photon<double>(qed_ctx *, const qed_species *, const qed_species *,
                                           const qed_species *, const int64_t *, const qed_fields *,
                                           int64_t, cudaStream_t);
template cudaError_t launch_compact<float>(qed_ctx *, const qed_species *, cudaStream_t);
template cudaError_t launch_compact<double>(qed_ctx *, const qed_species *, cudaStream_t);
template cudaError_t launch_compact_fill<float>(qed_ctx *, const qed_species *, cudaStream_t);
template cudaError_t launch_compact_fill<double>(qed_ctx *, const qed_species *, cudaStream_t);
template cudaError_t launch_eval<float>(qed_ctx *, int, int, const double *, const double *,
                                        const uint32_t *, double *, int64_t, cudaStream_t);
template cudaError_t launch_eval<double>(qed_ctx *, int, int, const double *, const double *,
                                         const uint32_t *, double *, int64_t, cudaStream_t);

}  // namespace qed
