// qed_onepass.cu -- the lepton step in a single pass, with photons appended in
// no particular order (qed_config.append_order = QED_APPEND_ANY, FP32 contexts,
// event generator Method I).
//
// What is computed is the ordered path's: per lepton, field gather, Boris
// push, chi_e (Eq. 2), W_rad (Eq. 1 above the xi_min cut), N = max(1,
// ceil(W Dt / 0.2)) sub-steps of Method I with Philox draws keyed by (id,
// step, sub-step / 2) -- one draw serves two sub-steps --, xi from the inverse
// CDF (Eq. 7) on an event, the recoil and the photon.  Every particle, photon id and photon energy is the same as
// on the ordered path; only the order of the appended photons differs (it
// depends on the scheduling of the warps), so the photon buffer is the same
// set in another order.
//
// How the work is laid out, per warp of a persistent grid:
//   streaming: each lane takes one particle of a 32-particle slice (the next
//     slice's words are in flight into shared memory, cp.async), pushes it and
//     computes chi.  The rate bound W <= w_j chi / gamma (w_j = alpha a_S
//     times the largest value of int_0^1 dW/dxi / chi in the rate table at
//     and above the row j at or below ln chi, so it holds with the xi_min cut)
//     settles most particles without the 2-D tables: if w_j chi Dt / gamma <=
//     0.2 the particle has one sub-step, and if its first draw r1 is not
//     below that bound it has no event -- it is finished (its pushed state
//     written).  The others go
//     to the warp's queue in shared memory (pushed momentum, fields, id,
//     slot).
//   heavy phase: when the queue holds 32 particles (a scheduling parameter,
//     as are the lane counts below), the warp runs them with
//     a per-warp scheduler of lane states -- idle; rate (chi and the exact
//     rate, and N for a new particle; idle lanes are refilled from the queue
//     at the start of such a round); scanning (Method I draws, four per
//     iteration from two independent Philox calls, up to 8 per round, the
//     round ending early when fewer than 8 lanes are still drawing); or pending (an
//     event; the emitting lanes run together: xi, the recoil, the photon;
//     then the rate again for the remaining sub-steps).  An
//     emission round reserves slots for its photons with one atomic on the
//     photon count and writes them there.  A round runs only when enough
//     lanes are in its state (16 for an emission, 12 otherwise); when none can,
//     the warp goes back to streaming and the chains still running are parked
//     in shared memory, to be resumed (with new entries) by the next heavy
//     phase.  After the last slice the queue is drained.
//   learned sampler: an event of a one-sub-step lepton inside the network's
//     domain ends its chain with a 16-byte record instead of an emission; the
//     dense pass k_net_emit (below) finishes those emissions, 32 per warp.
// No particle waits on another and nothing is staged in global memory: a
// particle is read once and its slot written once or twice (the pushed state,
// then the recoiled momentum of one that emitted, shortly after, while the
// line is still in L2).
#include <cstdio>

#include "qed_internal.h"
#include "qed_kernels.cuh"
#include "qed_mlp.cuh"

namespace qed {

namespace {

// CTAs of 4 warps: with the per-warp shared memory below, 5 fit on an SM
constexpr int OP_THREADS = 128;
constexpr int OP_WARPS = OP_THREADS / 32;
constexpr int QCAP = 64;       // queue entries per warp
constexpr int QEXIT = QCAP - 32;  // a heavy phase may end once the queue holds at most this many
constexpr int QF = 9;          // queue floats per entry: px py pz ex ey ez bx by bz
constexpr int PF = 17;         // parked floats per lane
constexpr int PU = 9;          // parked words per lane

struct OnePassArgs {
  Sp<float> sp[2];
  int nsp;
  Sp<float> ph;
  Fld<float> f;
  Consts C;
  Tables<float> T;
  Out o;
  int64_t step;
  const int64_t *d_step;
  const float *w_up_row;       // W_rad <= w_up_row[j] chi / gamma for ln chi >= row j
  float chi_tab_lo, chi_tab_hi;  // chi range of the rate tables
  const uint32_t *mlp_frag;  // learned sampler: BF16 fragments and the FP32 small
  const float *mlp_fw;       // layers, in global memory (read through L1)
  float4 *net_rec;           // records of the deferred network emissions
  unsigned long long *net_n; // their count
  int64_t net_cap;
  // chain scheduling (QED_SCHED_*): an emission round waits for emit_lanes
  // lanes with an event, a rate or scanning round runs with at least
  // round_lanes lanes, a scanning round draws scan_iters times four
  // sub-steps per lane and ends early when fewer than scan_left lanes are
  // still drawing; a heavy phase starts when the queue holds qtrig entries
  // (qtrig - 1 + 32 <= QCAP)
  int emit_lanes, round_lanes, scan_iters, scan_left, qtrig;
};

// dynamic shared memory: prefetch buffers, per-warp queues and park areas.
// The rate tables are read through L1: only the queued particles evaluate the
// exact rate.
template <int FM> __host__ __device__ size_t onepass_layout(const OnePassArgs &a, size_t off[4]) {
  size_t o = 0;
  off[0] = o;  // prefetch: two buffers of [NV][OP_THREADS] words and [OP_THREADS] ids
  o += 2 * OP_THREADS * ((size_t)stream_words<FM>() * sizeof(float) + sizeof(uint64_t));
  off[1] = o;  // queues: slot [QCAP], floats [QF][QCAP], ids [QCAP] per warp
  o += (size_t)OP_WARPS * QCAP * (4 + 4 * QF + 8);
  off[2] = o;  // park: floats [PF][32], words [PU][32] per warp
  o += (size_t)OP_WARPS * 32 * 4 * (PF + PU);
  o = (o + 15) & ~(size_t)15;
  off[3] = o;
  return o;
}

// lane states of a chain
enum { ST_IDLE = 0, ST_RATE = 1, ST_SCAN = 2, ST_PEND = 3, ST_DONE = 4 };

// Learned-sampler emissions deferred to the dense pass: one record per
// emission, 16 bytes -- the lepton's index (species in the top bit) and kappa
// -- plus, with grid fields, its position before the push (so that the dense
// pass gathers the same fields), 32 bytes.  Everything else (the pushed
// momentum, gamma, the direction, chi, the id) the dense pass reads or
// recomputes with the same expressions.
template <int FM> __host__ __device__ constexpr int net_stride() { return FM == FM_GRID ? 3 : 1; }  // float4 per record

// gamma and the unit direction of a pushed momentum, as a deferred particle
// gets them in the heavy phase and in the dense pass alike
__device__ __forceinline__ void gamma_dir(float px, float py, float pz, float &g, float &nx, float &ny,
                                          float &nz) {
  g = sqrtf(1.f + px * px + py * py + pz * pz);
  const float pm = sqrtf(px * px + py * py + pz * pz);
  nx = ny = nz = 0.f;
  if (pm > 0.f) {
    const float ip = 1.f / pm;
    nx = px * ip; ny = py * ip; nz = pz * ip;
  }
}


// N = max(1, ceil(W Dt / wdt_max)), capped at max_substeps (status bit).
__device__ __forceinline__ int64_t substep_count_op(const Consts &C, float W, float dt, float wdt_max,
                                                    uint32_t &status) {
  const float wdt = W * dt;
  if (!(wdt > wdt_max)) return 1;
  float nn = ceilf(wdt / wdt_max);
  if (nn > (float)C.max_substeps) {
    nn = (float)C.max_substeps;
    status |= QED_STATUS_SUBSTEPS;
  }
  return (int64_t)nn;
}

// DEF: the default chain scheduling as compile-time constants (the runtime
// values cost ~3.5% of the kernel's time); otherwise the values in A.
template <int FM, int MODE, bool MLP, bool DEF>
__global__ void __launch_bounds__(OP_THREADS, 5) k_lepton_onepass(OnePassArgs A) {
  const int emit_lanes = DEF ? SCHED_DEF_EMIT_LANES : A.emit_lanes;
  const int round_lanes = DEF ? SCHED_DEF_ROUND_LANES : A.round_lanes;
  const int scan_iters = DEF ? (SCHED_DEF_SCAN_DRAWS + 3) / 4 : A.scan_iters;
  const int scan_left = DEF ? SCHED_DEF_SCAN_LEFT : A.scan_left;
  const int qtrig = DEF ? SCHED_DEF_QUEUE_TRIGGER : A.qtrig;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ BlockTally bt;
  __shared__ long long s_meta[4];
  __shared__ unsigned long long s_deferred;
  constexpr int NV = stream_words<FM>();
  const int64_t step_ = A.d_step ? *A.d_step : A.step;
  size_t off[4];
  onepass_layout<FM>(A, off);
  const float *sR = A.T.R, *sF = A.T.F;
  float *pf = reinterpret_cast<float *>(smem_raw + off[0]);
  uint64_t *pf_id = reinterpret_cast<uint64_t *>(pf + 2 * NV * OP_THREADS);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;  // wid < OP_WARPS
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned char *qbase = smem_raw + off[1] + (size_t)wid * QCAP * (4 + 4 * QF + 8);
  uint32_t *q_slot = reinterpret_cast<uint32_t *>(qbase);
  float *q_f = reinterpret_cast<float *>(qbase + 4 * QCAP);
  uint64_t *q_id = reinterpret_cast<uint64_t *>(qbase + 4 * QCAP + 4 * QF * QCAP);
  unsigned char *pbase = smem_raw + off[2] + (size_t)wid * 32 * 4 * (PF + PU);
  float *pk_f = reinterpret_cast<float *>(pbase);
  uint32_t *pk_u = reinterpret_cast<uint32_t *>(pbase + 4 * PF * 32);
  block_tally_init(&bt);
  if (threadIdx.x == 0) {
    s_meta[0] = *(volatile int64_t *)A.sp[0].d_n;
    s_meta[1] = A.nsp > 1 ? *(volatile int64_t *)A.sp[1].d_n : 0;
    s_meta[2] = (long long)A.o.scan.sync[2];
    s_deferred = 0;
  }
  __syncthreads();
  const int64_t n0 = s_meta[0], n1 = s_meta[1];
  const uint32_t epoch = (uint32_t)s_meta[2];
  const int64_t T0 = (n0 + TILE - 1) / TILE, T1 = (n1 + TILE - 1) / TILE;
  const int64_t nslots = (T0 + T1) * TILE;
  const float inv_aS = A.C.f_inv_aS, dt = A.C.f_dt, wdt_max = A.C.f_wdt_max;
  Tally tl;
  tl.clear();
  uint32_t deferred = 0;  // heavy particles taken by this lane
  int qn = 0;             // queue length (warp-uniform)
  unsigned parked = 0;    // lanes with a parked chain (warp-uniform)

  auto slot_index = [&](int64_t sl, int &si, int64_t &i) {
    const int64_t tile = sl / TILE;
    si = tile < T0 ? 0 : 1;
    i = (tile - (si ? T0 : 0)) * TILE + (sl % TILE);
  };

  // ---- heavy phase: the queued particles' Method I chains ---------------
  // Lane states: idle; rate (chi and the exact rate due: a new particle or a
  // recoiled one); scan (drawing sub-steps); pend (an event, emission due).
  auto heavy_phase = [&](bool final_drain) {
    int st = ST_IDLE;
    uint32_t hslot = 0, wy = 0, cnt = 0;
    int N = 1, k = 0;
    float px = 0.f, py = 0.f, pz = 1.f, g = 1.f, chi = 0.f, dts = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
    float E[3] = {0.f, 0.f, 0.f}, B[3] = {0.f, 0.f, 0.f};
    RateOut<float> ro{0.f, -1e30f, 0.f};
    uint64_t pid = 0;
    if (parked & (1u << lane)) {  // resume a parked chain
      px = pk_f[0 * 32 + lane]; py = pk_f[1 * 32 + lane]; pz = pk_f[2 * 32 + lane];
      g = pk_f[3 * 32 + lane]; chi = pk_f[4 * 32 + lane]; dts = pk_f[5 * 32 + lane];
      ro.W = pk_f[6 * 32 + lane]; ro.kmin = pk_f[7 * 32 + lane]; ro.l = pk_f[8 * 32 + lane];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        E[c] = pk_f[(9 + c) * 32 + lane];
        B[c] = pk_f[(12 + c) * 32 + lane];
      }
      st = (int)pk_u[0 * 32 + lane];
      hslot = pk_u[1 * 32 + lane];
      N = (int)pk_u[2 * 32 + lane];
      k = (int)pk_u[3 * 32 + lane];
      wy = pk_u[4 * 32 + lane];
      cnt = pk_u[5 * 32 + lane];
      pid = (uint64_t)pk_u[6 * 32 + lane] | ((uint64_t)pk_u[7 * 32 + lane] << 32);
      nx = pk_f[15 * 32 + lane]; ny = pk_f[16 * 32 + lane];
      nz = __uint_as_float(pk_u[8 * 32 + lane]);
    }
    parked = 0;
    for (;;) {
      const unsigned idle = __ballot_sync(0xFFFFFFFFu, st == ST_IDLE);
      const unsigned rate = __ballot_sync(0xFFFFFFFFu, st == ST_RATE);
      const unsigned scan = __ballot_sync(0xFFFFFFFFu, st == ST_SCAN);
      const unsigned pend = __ballot_sync(0xFFFFFFFFu, st == ST_PEND);
      const int ni = __popc(idle), nr = __popc(rate), ns = __popc(scan), np = __popc(pend);
      // idle lanes are refilled from the queue at the start of a rate round
      const int take = min(qn, ni);
      // a round runs only with enough lanes in its state; otherwise the warp
      // goes back to streaming (once the queue has room for another slice)
      // and the chains wait, parked, for the next heavy phase -- except in
      // the final drain, which runs whatever is left
      int phase;
      if (np >= emit_lanes) phase = ST_PEND;
      else if (nr + take >= round_lanes) phase = ST_RATE;
      else if (ns >= round_lanes) phase = ST_SCAN;
      else if (!final_drain && qn <= QEXIT) break;
      else if (nr + take) phase = ST_RATE;
      else if (ns) phase = ST_SCAN;
      else if (np) phase = ST_PEND;
      else break;
      if (phase == ST_RATE) {
        // refill: idle lanes take queue entries from the top, in lane order
        if (st == ST_IDLE) {
          const int r = __popc(idle & lt_mask);
          if (r < take) {
            const int q = qn - 1 - r;
            hslot = q_slot[q];
            px = q_f[0 * QCAP + q]; py = q_f[1 * QCAP + q]; pz = q_f[2 * QCAP + q];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              E[c] = q_f[(3 + c) * QCAP + q];
              B[c] = q_f[(6 + c) * QCAP + q];
            }
            pid = q_id[q];
            gamma_dir(px, py, pz, g, nx, ny, nz);
            k = 0;
            cnt = 0;
            st = ST_RATE;
          }
        }
        qn -= take;
        // chi (Eq. 2) and the exact rate; a new particle also gets N
        if (st == ST_RATE) {
          chi = chi_lepton(px, py, pz, g, E[0], E[1], E[2], B[0], B[1], B[2], inv_aS);
          ro = photon_rate(sR, sF, A.T, A.C, chi, g, tl);
          if (k == 0 && cnt == 0) {
            N = (int)substep_count_op(A.C, ro.W, dt, wdt_max, tl.status);
            tl.substeps += N;
            dts = dt / (float)N;
            deferred += 1;
          }
          st = ST_SCAN;
        }
      } else if (phase == ST_SCAN) {
        // draws two sub-steps at a time (independent Philox chains run
        // interleaved; the second is used only if the first has no event),
        // for as long as enough lanes are still drawing: the others keep
        // their state for a later round
        const float thr = ro.W * dts;
        const bool was_scan = st == ST_SCAN;
        bool drawing = was_scan;
        for (int it = 0; it < scan_iters; ++it) {
          if (drawing) {
            // sub-steps 2j .. 2j+3 from the draws j and j+1 (words 0-1 and
            // 2-3 of each); a chain at an odd sub-step starts at 2j+1
            const int64_t j = k >> 1;
            const U4 ra = draw(A.C, pid, step_, j, STREAM_EMIT);
            const U4 rb = draw(A.C, pid, step_, j + 1, STREAM_EMIT);
            const uint32_t w1[4] = {ra.x, ra.z, rb.x, rb.z}, w2[4] = {ra.y, ra.w, rb.y, rb.w};
            const int q0 = (int)(k & 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (q >= q0 && st == ST_SCAN) {
                if (thr > unif<float>(w1[q])) { wy = w2[q]; st = ST_PEND; }
                else if (++k >= N) { st = ST_DONE; }
              }
            }
            drawing = st == ST_SCAN;
          }
          if (__popc(__ballot_sync(0xFFFFFFFFu, drawing)) < scan_left) break;
        }
        if (MLP) {
          // an event of a one-sub-step particle inside the network's domain
          // takes its xi from the learned sampler, in the dense pass that
          // follows this kernel: a record here (one per such particle: at
          // most n0 + n1, which the records hold), no photon yet (cnt = 0)
          bool net = false;
          float kap = 0.f;
          if (was_scan && st == ST_PEND && N == 1) {
            kap = photon_kappa(ro.kmin, unif<float>(wy), unif<float>(~wy));
            const float lchi = chi > 0.f ? logf(chi) : MLP_L_LO - 1.f;
            net = lchi >= MLP_L_LO && lchi <= MLP_L_HI && kap >= MLP_K_LO && kap <= MLP_K_HI;
          }
          const unsigned nm = __ballot_sync(0xFFFFFFFFu, net);
          if (nm) {
            const int leader = __ffs(nm) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(A.net_n, (unsigned long long)__popc(nm));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (net) {
              constexpr int RS = net_stride<FM>();
              const unsigned long long r = base + __popc(nm & lt_mask);
              if (r < (unsigned long long)(A.net_cap / RS)) {
                int si;
                int64_t i;
                slot_index(hslot, si, i);
                float4 *R = A.net_rec + RS * r;
                R[0] = make_float4(__uint_as_float((uint32_t)i),
                                   __uint_as_float((uint32_t)((uint64_t)i >> 32) | ((uint32_t)si << 31)),
                                   kap, E[0]);
                if (FM == FM_GRID) {
                  R[1] = make_float4(E[1], E[2], B[0], B[1]);
                  R[2] = make_float4(B[2], 0.f, 0.f, 0.f);
                }
              } else {  // only with counts beyond the species' capacities
                tl.dropped += 1;
                tl.status |= QED_STATUS_CAPACITY;
              }
              st = ST_DONE;
            }
          }
        }
      } else {
        // emission by every lane with an event: kappa and ln delta from the
        // inverse table (Eq. 7), xi, the recoil and the photon
        const bool ev = st == ST_PEND;
        const float kap = ev ? photon_kappa(ro.kmin, unif<float>(wy), unif<float>(~wy)) : 0.f;
        float eph = 0.f, g2 = g;
        if (ev) {
          const float Y = photon_lndelta_table(A.T.Y, A.T, ro.l, kap, tl);
          const XiOut<float> xo = xi_from_lndelta(chi, Y);
          g2 = g * xo.omxi;
          eph = g * xo.xi;
          if (g2 < 1.f) { g2 = 1.f; eph = g - 1.f; }
          const int b = spec_bin(A.C, eph);
          const unsigned em = __activemask();
          const unsigned same = __match_any_sync(em, b);
          if (b >= 0 && lane == __ffs(same) - 1) atomicAdd(&bt.hist[b], (unsigned long long)__popc(same));
        }
        // photon slots: one atomic per emission round
        const unsigned em = __ballot_sync(0xFFFFFFFFu, ev);
        const int leader = __ffs(em) - 1;
        unsigned long long base = 0;
        if (lane == leader)
          base = atomicAdd(reinterpret_cast<unsigned long long *>(A.ph.d_n), (unsigned long long)__popc(em));
        base = __shfl_sync(0xFFFFFFFFu, base, leader < 0 ? 0 : leader);
        if (ev) {
          const int64_t pos = (int64_t)base + __popc(em & lt_mask);
          if (pos >= A.ph.cap) {
            tl.dropped += 1;
            tl.status |= QED_STATUS_CAPACITY;
          } else {
            int si;
            int64_t i;
            slot_index(hslot, si, i);
            const Sp<float> &S = A.sp[si];
            const U4 cid = draw(A.C, pid, step_, k, STREAM_PHOTON_ID);
            write_child(A.ph, pos, S.x[i], S.y[i], S.z[i], eph * nx, eph * ny, eph * nz, S.w[i],
                        (uint64_t)cid.x | ((uint64_t)cid.y << 32), E, B, S.tag ? S.tag[i] : 0u);
          }
          ++cnt;
          const float pm2 = sqrtf((g2 - 1.f) * (g2 + 1.f));
          px = pm2 * nx; py = pm2 * ny; pz = pm2 * nz;
          g = g2;
          // the rate for the remaining sub-steps, or the end of the chain
          st = ++k >= N ? ST_DONE : ST_RATE;
        }
      }
      // the end of a chain: the recoiled momentum of a particle that emitted
      if (st == ST_DONE) {
        if (cnt > 0) {
          int si;
          int64_t i;
          slot_index(hslot, si, i);
          const Sp<float> &S = A.sp[si];
          const float pm = sqrtf((g - 1.f) * (g + 1.f));
          S.px[i] = pm * nx; S.py[i] = pm * ny; S.pz[i] = pm * nz;
        }
        tl.events += cnt;
        st = ST_IDLE;
      }
    }
    // park the chains still running
    parked = __ballot_sync(0xFFFFFFFFu, st != ST_IDLE);
    if (st != ST_IDLE) {
      pk_f[0 * 32 + lane] = px; pk_f[1 * 32 + lane] = py; pk_f[2 * 32 + lane] = pz;
      pk_f[3 * 32 + lane] = g; pk_f[4 * 32 + lane] = chi; pk_f[5 * 32 + lane] = dts;
      pk_f[6 * 32 + lane] = ro.W; pk_f[7 * 32 + lane] = ro.kmin; pk_f[8 * 32 + lane] = ro.l;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pk_f[(9 + c) * 32 + lane] = E[c];
        pk_f[(12 + c) * 32 + lane] = B[c];
      }
      pk_f[15 * 32 + lane] = nx;
      pk_f[16 * 32 + lane] = ny;
      pk_u[0 * 32 + lane] = (uint32_t)st;
      pk_u[1 * 32 + lane] = hslot;
      pk_u[2 * 32 + lane] = (uint32_t)N;
      pk_u[3 * 32 + lane] = (uint32_t)k;
      pk_u[4 * 32 + lane] = wy;
      pk_u[5 * 32 + lane] = cnt;
      pk_u[6 * 32 + lane] = (uint32_t)pid;
      pk_u[7 * 32 + lane] = (uint32_t)(pid >> 32);
      pk_u[8 * 32 + lane] = __float_as_uint(nz);
    }
    __syncwarp();
  };

  // ---- streaming over all leptons, with the heavy phase in between -------
  // Each lane copies its next particle's words into shared memory with
  // asynchronous copies (cp.async) while the current one computes.  (One-
  // dimensional bulk copies of a warp's 128-byte slice of each array, issued
  // by one lane and completed on an mbarrier, measured slower: 3.98 against
  // 3.25 ms per step at 64M electrons.)
  const int t = threadIdx.x;
  auto prefetch = [&](int64_t sl, int b) {
    int si;
    int64_t i;
    slot_index(sl, si, i);
    const Sp<float> &S = A.sp[si];
    if (i >= (si ? n1 : n0)) return;
    float *d = pf + (size_t)b * NV * OP_THREADS + t;
    const float *src[12] = {S.x, S.y, S.z, S.px, S.py, S.pz, S.ex, S.ey, S.ez, S.bx, S.by, S.bz};
#pragma unroll
    for (int c = 0; c < NV; ++c) cp_async<4>(d + c * OP_THREADS, src[c] + i);
    cp_async<8>(pf_id + b * OP_THREADS + t, S.id + i);
  };
  const int64_t stride = (int64_t)gridDim.x * OP_THREADS;
  int buf = 0;
  int64_t slot = blockIdx.x * (int64_t)OP_THREADS + threadIdx.x;
  if (slot < nslots) prefetch(slot, 0);
  cp_async_commit();
  // nslots is a multiple of OP_THREADS: every lane of a warp runs the same
  // iterations; the one call of the heavy phase keeps its code once
  for (;;) {
    const bool streaming = slot < nslots;
    if (streaming) {
      if (slot + stride < nslots) prefetch(slot + stride, buf ^ 1);
      cp_async_commit();
      cp_async_wait<1>();
      int si;
      int64_t i;
      slot_index(slot, si, i);
      const Sp<float> &S = A.sp[si];
      bool heavy = false;
      float px = 0.f, py = 0.f, pz = 0.f;
      float E[3] = {0.f, 0.f, 0.f}, B[3] = {0.f, 0.f, 0.f};
      uint64_t pid = 0;
      if (i < (si ? n1 : n0)) {
        const float *v = pf + (size_t)buf * NV * OP_THREADS + t;
        float x = v[0], y = v[OP_THREADS], z = v[2 * OP_THREADS];
        px = v[3 * OP_THREADS]; py = v[4 * OP_THREADS]; pz = v[5 * OP_THREADS];
        if (FM == FM_PER_PARTICLE) {
          E[0] = v[6 * OP_THREADS]; E[1] = v[7 * OP_THREADS]; E[2] = v[8 * OP_THREADS];
          B[0] = v[9 * OP_THREADS]; B[1] = v[10 * OP_THREADS]; B[2] = v[11 * OP_THREADS];
        } else {
          get_fields<float, FM>(S, A.f, i, x, y, z, E, B);
        }
        pid = pf_id[buf * OP_THREADS + t];
        float g;
        if (MODE != MODE_EMIT) {
          g = boris(px, py, pz, E, B, S.q, dt);
          const float ig = r_div(dt, g);
          x += px * ig; y += py * ig; z += pz * ig;
        } else {
          g = sqrtf(1.f + px * px + py * py + pz * pz);
        }
        if (!(g < 1e30f)) {
          tl.status |= QED_STATUS_NONFINITE;  // left as it was
        } else {
          const float chi = chi_lepton(px, py, pz, g, E[0], E[1], E[2], B[0], B[1], B[2], inv_aS);
          // one sub-step and no event, for sure, from the rate bound of the
          // table row at or below ln chi, and r1
          const float fj = (r_log(chi) - A.T.gl.x0) * A.T.gl.inv_h;
          const int j = fj >= 0.f ? (fj < (float)(A.T.gl.n - 1) ? (int)fj : A.T.gl.n - 1) : 0;
          const float wdt_up = r_div(__ldg(A.w_up_row + j) * dt * chi, g);
          bool done = false;
          if (wdt_up <= wdt_max) {
            const U4 r = draw(A.C, pid, step_, 0, STREAM_EMIT);
            done = !(wdt_up > unif<float>(r.x));
          }
          if (done) {
            tl.substeps += 1;
            if (chi > 0.f && (chi < A.chi_tab_lo || chi > A.chi_tab_hi)) {
              tl.domain += 1;
              tl.status |= QED_STATUS_DOMAIN;
            }
          } else {
            heavy = true;
          }
          if (MODE != MODE_EMIT) {
            S.x[i] = x; S.y[i] = y; S.z[i] = z;
            S.px[i] = px; S.py[i] = py; S.pz[i] = pz;
          }
        }
      }
      const unsigned hm = __ballot_sync(0xFFFFFFFFu, heavy);
      if (heavy) {
        const int q = qn + __popc(hm & lt_mask);
        q_slot[q] = (uint32_t)slot;
        q_f[0 * QCAP + q] = px; q_f[1 * QCAP + q] = py; q_f[2 * QCAP + q] = pz;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          q_f[(3 + c) * QCAP + q] = E[c];
          q_f[(6 + c) * QCAP + q] = B[c];
        }
        q_id[q] = pid;
      }
      qn += __popc(hm);
      slot += stride;
      buf ^= 1;
    } else {
      cp_async_wait<0>();
    }
    if (qn >= qtrig || !streaming) {
      __syncwarp();  // queue entries and the pushed state written above are visible to the warp
      heavy_phase(!streaming);
    }
    if (!streaming) break;
  }

  tally_flush(&bt, tl);
  {
    uint32_t d = deferred;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xFFFFFFFFu, d, o);
    if (lane == 0 && d) atomicAdd(&s_deferred, (unsigned long long)d);
  }
  __syncthreads();
  block_tally_commit(&bt, A.o.cnt, 0);
  if (threadIdx.x == 0) {
    if (s_deferred) atomicAdd(reinterpret_cast<unsigned long long *>(&A.o.cnt->deferred), s_deferred);
    // the last CTA to finish clamps the photon count to the capacity (the
    // slots past it were counted as dropped) and resets the shared counters
    __threadfence();
    const unsigned int prev = atomicAdd(&A.o.scan.sync[1], 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      int64_t *dn = A.ph.d_n;
      if (*(volatile int64_t *)dn > A.ph.cap) *dn = A.ph.cap;
      A.o.scan.sync[0] = 0u;
      A.o.scan.sync[1] = 0u;
      A.o.scan.sync[2] = epoch + 1u;
      __threadfence();
    }
  }
}

// ---- the learned sampler's dense pass ----------------------------------
// The deferred emissions of one-sub-step leptons (records written by the
// single-pass kernel): every warp takes 32 records at a time, evaluates the
// network for all of them at once (tensor cores, weights in shared memory),
// and finishes each emission with the heavy phase's expressions: gamma, the
// direction and chi of the pushed lepton, xi (Eq. 7 through ln delta), the
// recoiled momentum, the spectrum bin and the photon.
struct NetArgs {
  Sp<float> sp[2];
  Sp<float> ph;
  Fld<float> f;
  Consts C;
  Out o;
  int64_t step;
  const int64_t *d_step;
  const uint32_t *mlp_frag;
  const float *mlp_fw;
  const float4 *net_rec;
  unsigned long long *net_n;  // [0] records written, [1] CTAs of this pass done
  int64_t net_cap;            // float4 units of net_rec
};
constexpr int NET_THREADS = 256;

template <int FM>
__global__ void __launch_bounds__(NET_THREADS) k_net_emit(NetArgs A) {
  constexpr int RS = net_stride<FM>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ BlockTally bt;
  __shared__ long long s_n;
  uint32_t *s_frag = reinterpret_cast<uint32_t *>(smem_raw);
  float *s_fw = reinterpret_cast<float *>(s_frag + MLP_FRAG_WORDS);
  for (int k = threadIdx.x; k < MLP_FRAG_WORDS; k += blockDim.x) s_frag[k] = A.mlp_frag[k];
  for (int k = threadIdx.x; k < MLP_SMEM_FLOATS; k += blockDim.x) s_fw[k] = A.mlp_fw[k];
  block_tally_init(&bt);
  if (threadIdx.x == 0) {
    const unsigned long long n = *(volatile unsigned long long *)A.net_n;
    const unsigned long long cap = (unsigned long long)(A.net_cap / RS);
    s_n = (long long)(n < cap ? n : cap);
  }
  __syncthreads();
  const int64_t n = s_n;
  const int64_t step_ = A.d_step ? *A.d_step : A.step;
  const float inv_aS = A.C.f_inv_aS;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  Tally tl;
  tl.clear();
  for (int64_t base = w * 32; base < n; base += nw * 32) {  // warp-uniform
    const int64_t r = base + lane;
    const bool ok = r < n;
    int si = 0;
    int64_t i = 0;
    float kap = 0.f, g = 1.f, nx = 0.f, ny = 0.f, nz = 0.f, chi = 1.f;
    float E[3] = {0.f, 0.f, 0.f}, B[3] = {0.f, 0.f, 0.f};
    if (ok) {
      const float4 *R = A.net_rec + RS * r;
      const float4 R0 = R[0];
      const uint32_t hi = __float_as_uint(R0.y);
      i = (int64_t)(((uint64_t)(hi & 0x7FFFFFFFu) << 32) | __float_as_uint(R0.x));
      si = (int)(hi >> 31);
      kap = R0.z;
      const Sp<float> &S = A.sp[si];
      if (FM == FM_GRID) {
        const float4 R1 = R[1], R2 = R[2];
        E[0] = R0.w; E[1] = R1.x; E[2] = R1.y;
        B[0] = R1.z; B[1] = R1.w; B[2] = R2.x;
      } else {
        get_fields<float, FM>(S, A.f, i, 0.f, 0.f, 0.f, E, B);
      }
      const float px = S.px[i], py = S.py[i], pz = S.pz[i];
      gamma_dir(px, py, pz, g, nx, ny, nz);
      chi = chi_lepton(px, py, pz, g, E[0], E[1], E[2], B[0], B[1], B[2], inv_aS);
    }
    const float lchi = ok ? logf(chi) : 0.f;
    const float zz = mlp_infer_warp(s_frag, s_fw, (lchi - MLP_LC) / MLP_LS, (kap - MLP_KC) / MLP_KS);
    float eph = 0.f, g2 = g;
    if (ok) {
      const float Y = zz + mlp_baseline(kap);
      const XiOut<float> xo = xi_from_lndelta(chi, Y);
      g2 = g * xo.omxi;
      eph = g * xo.xi;
      if (g2 < 1.f) { g2 = 1.f; eph = g - 1.f; }
      const int b = spec_bin(A.C, eph);
      const unsigned same = __match_any_sync(__activemask(), b);
      if (b >= 0 && lane == __ffs(same) - 1) atomicAdd(&bt.hist[b], (unsigned long long)__popc(same));
    }
    const unsigned em = __ballot_sync(0xFFFFFFFFu, ok);
    const int leader = __ffs(em) - 1;
    unsigned long long pbase = 0;
    if (lane == leader)
      pbase = atomicAdd(reinterpret_cast<unsigned long long *>(A.ph.d_n), (unsigned long long)__popc(em));
    pbase = __shfl_sync(0xFFFFFFFFu, pbase, leader < 0 ? 0 : leader);
    if (ok) {
      const Sp<float> &S = A.sp[si];
      const int64_t pos = (int64_t)pbase + __popc(em & lt_mask);
      if (pos >= A.ph.cap) {
        tl.dropped += 1;
        tl.status |= QED_STATUS_CAPACITY;
      } else {
        const U4 cid = draw(A.C, S.id[i], step_, 0, STREAM_PHOTON_ID);
        write_child(A.ph, pos, S.x[i], S.y[i], S.z[i], eph * nx, eph * ny, eph * nz, S.w[i],
                    (uint64_t)cid.x | ((uint64_t)cid.y << 32), E, B, S.tag ? S.tag[i] : 0u);
      }
      const float pm = sqrtf((g2 - 1.f) * (g2 + 1.f));
      S.px[i] = pm * nx; S.py[i] = pm * ny; S.pz[i] = pm * nz;
      tl.events += 1;
    }
  }
  tally_flush(&bt, tl);
  __syncthreads();
  block_tally_commit(&bt, A.o.cnt, 0);
  if (threadIdx.x == 0) {
    // the last CTA clamps the photon count to the capacity and clears the
    // record count for the next step
    __threadfence();
    const unsigned long long prev = atomicAdd(A.net_n + 1, 1ull);
    if (prev == gridDim.x - 1) {
      __threadfence();
      int64_t *dn = A.ph.d_n;
      if (*(volatile int64_t *)dn > A.ph.cap) *dn = A.ph.cap;
      A.net_n[0] = 0ull;
      A.net_n[1] = 0ull;
      __threadfence();
    }
  }
}

template <int FM>
cudaError_t launch_net_emit_t(qed_ctx *c, const NetArgs &n, cudaStream_t st) {
  const size_t sm = MLP_SMEM_BYTES;
  auto kern = k_net_emit<FM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NET_THREADS, sm);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_COMPACT);
  kern<<<c->num_sms * per_sm, NET_THREADS, sm, st>>>(n);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_net_emit(qed_ctx *c, const OnePassArgs &a, int fm, cudaStream_t st) {
  NetArgs n{};
  n.sp[0] = a.sp[0];
  n.sp[1] = a.nsp > 1 ? a.sp[1] : a.sp[0];
  n.ph = a.ph;
  n.f = a.f;
  n.C = a.C;
  n.o = a.o;
  n.step = a.step;
  n.d_step = a.d_step;
  n.mlp_frag = a.mlp_frag;
  n.mlp_fw = a.mlp_fw;
  n.net_rec = a.net_rec;
  n.net_n = a.net_n;
  n.net_cap = a.net_cap;
  if (fm == QED_FIELDS_UNIFORM) return launch_net_emit_t<FM_UNIFORM>(c, n, st);
  if (fm == QED_FIELDS_PER_PARTICLE) return launch_net_emit_t<FM_PER_PARTICLE>(c, n, st);
  return launch_net_emit_t<FM_GRID>(c, n, st);
}

template <int FM, int MODE, bool MLP>
cudaError_t launch_onepass_t(qed_ctx *c, const OnePassArgs &a, cudaStream_t st) {
  size_t off[4];
  const size_t sm = onepass_layout<FM>(a, off);
  bool dflt = true;
  for (int k = 0; k < QED_SCHED_PARAMS; ++k) dflt = dflt && sched_param(c, k) == sched_default(k);
  auto kern = dflt ? k_lepton_onepass<FM, MODE, MLP, true> : k_lepton_onepass<FM, MODE, MLP, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, OP_THREADS, sm);
  if (e != cudaSuccess) return e;
  per_sm = persistent_blocks_per_sm(c, per_sm, QED_TUNE_STREAM);
  kern<<<c->num_sms * per_sm, OP_THREADS, sm, st>>>(a);
  c->launches += 1;
  return cudaGetLastError();
}

template <int MODE, bool MLP>
cudaError_t launch_onepass_m(qed_ctx *c, const OnePassArgs &a, int fm, cudaStream_t st) {
  if (fm == QED_FIELDS_UNIFORM) return launch_onepass_t<FM_UNIFORM, MODE, MLP>(c, a, st);
  if (fm == QED_FIELDS_PER_PARTICLE) return launch_onepass_t<FM_PER_PARTICLE, MODE, MLP>(c, a, st);
  return launch_onepass_t<FM_GRID, MODE, MLP>(c, a, st);
}

}  // namespace

// The lepton step of an unordered-append FP32 context (electrons s0 and, if
// given, positrons s1; photons appended to ph).  mode: 1 emission only
// (qed_emit), 2 push and emission (qed_step_fused).
cudaError_t launch_lepton_onepass(qed_ctx *c, const qed_species *s0, const qed_species *s1,
                                  const qed_species *ph, const qed_fields *f, int64_t step,
                                  int mode, cudaStream_t st) {
  OnePassArgs a{};
  a.sp[0] = to_sp<float>(s0);
  a.nsp = s1 ? 2 : 1;
  if (s1) a.sp[1] = to_sp<float>(s1);
  a.ph = to_sp<float>(ph);
  a.f = to_fld<float>(f);
  a.C = consts_of(c);
  a.T = tables_of<float>(c);
  a.o = out_of(c);
  a.step = step;
  a.d_step = c->use_dstep ? c->d_step : nullptr;
  a.w_up_row = c->w_up_row;
  a.chi_tab_lo = (float)exp(c->gl.lo);
  a.chi_tab_hi = (float)exp(c->gl.hi);
  a.mlp_frag = c->mlp_frag;
  a.mlp_fw = c->mlp_fw;
  a.net_rec = c->net_rec;
  a.net_n = c->net_n;
  a.net_cap = c->net_cap;
  a.emit_lanes = sched_param(c, QED_SCHED_EMIT_LANES);
  a.round_lanes = sched_param(c, QED_SCHED_ROUND_LANES);
  a.scan_iters = (sched_param(c, QED_SCHED_SCAN_DRAWS) + 3) / 4;
  a.scan_left = sched_param(c, QED_SCHED_SCAN_LEFT);
  a.qtrig = min(sched_param(c, QED_SCHED_QUEUE_TRIGGER), QCAP - 31);
  const bool mlp = c->cfg.sampler == QED_SAMPLER_MLP && c->mlp_ready && c->net_rec;
  cudaError_t e;
  if (mode == MODE_EMIT)
    e = mlp ? launch_onepass_m<MODE_EMIT, true>(c, a, f->mode, st)
            : launch_onepass_m<MODE_EMIT, false>(c, a, f->mode, st);
  else
    e = mlp ? launch_onepass_m<MODE_FUSED, true>(c, a, f->mode, st)
            : launch_onepass_m<MODE_FUSED, false>(c, a, f->mode, st);
  if (e == cudaSuccess) e = prof_mark(c, 1, st);
  if (e == cudaSuccess && mlp) e = launch_net_emit(c, a, f->mode, st);
  return e;
}

}  // namespace qed
