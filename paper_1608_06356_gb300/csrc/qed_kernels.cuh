// qed_kernels.cuh -- device building blocks shared by the step kernels of
// libqed (structure-of-arrays views, field gather, Boris push, block tallies,
// asynchronous copies, child writes) and the host helpers that build their
// arguments from the C ABI structs.
#pragma once
#include <cstdint>

#include "qed_internal.h"

namespace qed {

template <class Real> struct Sp {
  Real *x, *y, *z, *px, *py, *pz, *w;
  uint64_t *id;
  uint8_t *alive;
  Real *ex, *ey, *ez, *bx, *by, *bz;
  int64_t *d_n;
  int64_t cap;
  Real q;
  uint32_t *tag;  // optional, inherited by children
  Real *od_p, *od_r;  // event generators II/III: P_cum and r3 (0 = not drawn yet)
};

template <class Real> struct Fld {
  Real e[3], b[3];
  const float *grid;
  int nx, ny, nz;
  Real idx, idy, idz, x0, y0, z0;
};

enum { FM_UNIFORM = 0, FM_PER_PARTICLE = 1, FM_GRID = 2 };
enum { GEN_METHOD_I = 0, GEN_METHOD_II = 1, GEN_METHOD_III = 2 };
enum { MODE_PUSH = 0, MODE_EMIT = 1, MODE_FUSED = 2 };
// classes of the streaming lepton pass: 1 one sub-step with an event; 2-5 more
// than one sub-step, binned by N (<= 3, <= 7, <= 15, >= 16)
constexpr int NCLS = 5;

struct Out {
  qed_counters *cnt;
  ScanState scan;
};

// CIC gather from grid[nz][ny][nx][8] (periodic).
template <class Real>
__device__ __forceinline__ void cic_gather(const Fld<Real> &f, Real x, Real y, Real z, Real E[3],
                                           Real B[3]) {
  Real fx = (x - f.x0) * f.idx, fy = (y - f.y0) * f.idy, fz = (z - f.z0) * f.idz;
  Real ix = m_floor(fx), iy = m_floor(fy), iz = m_floor(fz);
  Real wx = fx - ix, wy = fy - iy, wz = fz - iz;
  long long i0 = (long long)ix, j0 = (long long)iy, k0 = (long long)iz;
  i0 %= f.nx; if (i0 < 0) i0 += f.nx;
  j0 %= f.ny; if (j0 < 0) j0 += f.ny;
  k0 %= f.nz; if (k0 < 0) k0 += f.nz;
  long long i1 = i0 + 1 == f.nx ? 0 : i0 + 1;
  long long j1 = j0 + 1 == f.ny ? 0 : j0 + 1;
  long long k1 = k0 + 1 == f.nz ? 0 : k0 + 1;
#pragma unroll
  for (int c = 0; c < 3; ++c) { E[c] = (Real)0; B[c] = (Real)0; }
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        Real w = (di ? wx : (Real)1 - wx) * (dj ? wy : (Real)1 - wy) * (dk ? wz : (Real)1 - wz);
        long long node = ((dk ? k1 : k0) * f.ny + (dj ? j1 : j0)) * f.nx + (di ? i1 : i0);
        const float4 *pn = reinterpret_cast<const float4 *>(f.grid + 8 * node);
        float4 a = __ldg(pn), b = __ldg(pn + 1);
        E[0] += w * (Real)a.x; E[1] += w * (Real)a.y; E[2] += w * (Real)a.z;
        B[0] += w * (Real)a.w; B[1] += w * (Real)b.x; B[2] += w * (Real)b.y;
      }
}

// Relativistic Boris push; returns gamma after the push.
template <class Real>
__device__ __forceinline__ Real boris(Real &px, Real &py, Real &pz, const Real E[3],
                                      const Real B[3], Real q, Real dt) {
  Real h = (Real)0.5 * q * dt;
  Real ux = px + h * E[0], uy = py + h * E[1], uz = pz + h * E[2];
  Real ig = h * r_rsqrt((Real)1 + ux * ux + uy * uy + uz * uz);  // h / gamma-
  Real tx = B[0] * ig, ty = B[1] * ig, tz = B[2] * ig;
  Real t2 = tx * tx + ty * ty + tz * tz;
  Real s = r_div((Real)2, (Real)1 + t2);
  Real sx = tx * s, sy = ty * s, sz = tz * s;
  Real vx = ux + (uy * tz - uz * ty), vy = uy + (uz * tx - ux * tz), vz = uz + (ux * ty - uy * tx);
  ux += vy * sz - vz * sy;
  uy += vz * sx - vx * sz;
  uz += vx * sy - vy * sx;
  px = ux + h * E[0];
  py = uy + h * E[1];
  pz = uz + h * E[2];
  return m_sqrt((Real)1 + px * px + py * py + pz * pz);
}

// ---------------------------------------------------------------------------
// block-level tallies
// ---------------------------------------------------------------------------
struct BlockTally {
  unsigned long long events, substeps, dropped, domain;
  unsigned int status;
  unsigned long long hist[64];
};

__device__ __forceinline__ void tally_flush(BlockTally *bt, const Tally &tl) {
  // warp reduce then one shared atomic per warp
  long long e = tl.events, s = tl.substeps, d = tl.dropped, m = tl.domain;
  unsigned st = tl.status;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
    s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    d += __shfl_xor_sync(0xFFFFFFFFu, d, o);
    m += __shfl_xor_sync(0xFFFFFFFFu, m, o);
    st |= __shfl_xor_sync(0xFFFFFFFFu, st, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (e) atomicAdd(&bt->events, (unsigned long long)e);
    if (s) atomicAdd(&bt->substeps, (unsigned long long)s);
    if (d) atomicAdd(&bt->dropped, (unsigned long long)d);
    if (m) atomicAdd(&bt->domain, (unsigned long long)m);
    if (st) atomicOr(&bt->status, st);
  }
}

__device__ __forceinline__ void block_tally_init(BlockTally *bt) {
  if (threadIdx.x == 0) {
    bt->events = bt->substeps = bt->dropped = bt->domain = 0;
    bt->status = 0;
  }
  for (int b = threadIdx.x; b < 64; b += blockDim.x) bt->hist[b] = 0;
}

// which: 0 -> emit_events, 1 -> pair_events
__device__ __forceinline__ void block_tally_commit(BlockTally *bt, qed_counters *g, int which) {
  if (threadIdx.x == 0) {
    unsigned long long *ev = reinterpret_cast<unsigned long long *>(which ? &g->pair_events
                                                                          : &g->emit_events);
    if (bt->events) atomicAdd(ev, bt->events);
    if (bt->substeps) atomicAdd(reinterpret_cast<unsigned long long *>(&g->substeps), bt->substeps);
    if (bt->dropped) atomicAdd(reinterpret_cast<unsigned long long *>(&g->dropped), bt->dropped);
    if (bt->domain) atomicAdd(reinterpret_cast<unsigned long long *>(&g->domain), bt->domain);
    if (bt->status) atomicOr(&g->status, bt->status);
  }
  for (int b = threadIdx.x; b < 64; b += blockDim.x)
    if (bt->hist[b]) atomicAdd(reinterpret_cast<unsigned long long *>(&g->hist[b]), bt->hist[b]);
}

// End of a persistent launch: the last CTA to finish resets the tile counter
// and advances the epoch for the next launch.
__device__ __forceinline__ void launch_epilogue(const ScanState &S, uint32_t epoch) {
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(&S.sync[1], 1u);
    if (prev == gridDim.x - 1) {
      S.sync[0] = 0u;
      S.sync[1] = 0u;
      S.sync[2] = epoch + 1u;
      __threadfence();
    }
  }
}

// Asynchronous global -> shared copies of one thread's own words (cp.async):
// the data of the next particle is in flight while the current one computes.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

template <class Real>
__device__ __forceinline__ void load_tables_smem(Real *dst, const Real *src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

template <class Real, int FM>
__device__ __forceinline__ void get_fields(const Sp<Real> &s, const Fld<Real> &f, int64_t i,
                                           Real x, Real y, Real z, Real E[3], Real B[3]) {
  if (FM == FM_UNIFORM) {
#pragma unroll
    for (int c = 0; c < 3; ++c) { E[c] = f.e[c]; B[c] = f.b[c]; }
  } else if (FM == FM_PER_PARTICLE) {
    E[0] = s.ex[i]; E[1] = s.ey[i]; E[2] = s.ez[i];
    B[0] = s.bx[i]; B[1] = s.by[i]; B[2] = s.bz[i];
  } else {
    cic_gather(f, x, y, z, E, B);
  }
}

template <class Real>
__device__ __forceinline__ int spec_bin(const Consts &C, Real eps) {
  const Real lo = sel<Real>(C.spec_lo, C.f_spec_lo);
  if (!(eps >= lo)) return -1;
  // (the FP32 path bins with the fast logarithm: a photon within ~1e-6 of a
  // bin edge may fall on either side, as it may against FP64 binning anyway)
  Real b = m_floor(sel<Real>(C.spec_scale, C.f_spec_scale) * r_log(r_div(eps, lo)));
  if (b < (Real)0 || b >= (Real)64) return -1;
  return (int)b;
}

template <class Real>
__device__ __forceinline__ void write_child(const Sp<Real> &d, int64_t slot, Real x, Real y, Real z,
                                            Real px, Real py, Real pz, Real w, uint64_t id,
                                            const Real E[3], const Real B[3], uint32_t tag) {
  d.x[slot] = x; d.y[slot] = y; d.z[slot] = z;
  d.px[slot] = px; d.py[slot] = py; d.pz[slot] = pz;
  d.w[slot] = w;
  d.id[slot] = id;
  if (d.tag) d.tag[slot] = tag;
  if (d.alive) d.alive[slot] = 1;
  if (d.od_p) { d.od_p[slot] = (Real)0; d.od_r[slot] = (Real)0; }
  if (d.ex) {
    d.ex[slot] = E[0]; d.ey[slot] = E[1]; d.ez[slot] = E[2];
    d.bx[slot] = B[0]; d.by[slot] = B[1]; d.bz[slot] = B[2];
  }
}

// Words a streaming kernel prefetches per particle: x, y, z, px, py, pz (+ E,
// B when the fields are per particle); the id goes to its own 8-byte slot.
// Two buffers (the slice being computed and the next one in flight).
template <int FM> __host__ __device__ constexpr int stream_words() { return FM == FM_PER_PARTICLE ? 12 : 6; }
template <class Real, int FM> __host__ __device__ constexpr size_t stream_prefetch_bytes() {
  return 2 * TILE * ((size_t)stream_words<FM>() * sizeof(Real) + sizeof(uint64_t));
}

// ---------------------------------------------------------------------------
// Host-side argument helpers
// ---------------------------------------------------------------------------
template <class Real> Sp<Real> to_sp(const qed_species *s) {
  Sp<Real> d{};
  if (!s) return d;
  d.x = (Real *)s->x; d.y = (Real *)s->y; d.z = (Real *)s->z;
  d.px = (Real *)s->px; d.py = (Real *)s->py; d.pz = (Real *)s->pz; d.w = (Real *)s->w;
  d.id = s->id; d.alive = s->alive;
  d.ex = (Real *)s->ex; d.ey = (Real *)s->ey; d.ez = (Real *)s->ez;
  d.bx = (Real *)s->bx; d.by = (Real *)s->by; d.bz = (Real *)s->bz;
  d.d_n = s->d_n; d.cap = s->capacity; d.q = (Real)s->q;
  d.tag = s->tag;
  d.od_p = (Real *)s->od_p; d.od_r = (Real *)s->od_r;
  return d;
}

template <class Real> Fld<Real> to_fld(const qed_fields *f) {
  Fld<Real> d{};
  for (int c = 0; c < 3; ++c) { d.e[c] = (Real)f->e[c]; d.b[c] = (Real)f->b[c]; }
  d.grid = f->grid;
  d.nx = f->nx; d.ny = f->ny; d.nz = f->nz;
  if (f->mode == QED_FIELDS_GRID) {
    d.idx = (Real)(1.0 / f->dx); d.idy = (Real)(1.0 / f->dy); d.idz = (Real)(1.0 / f->dz);
  }
  d.x0 = (Real)f->x0; d.y0 = (Real)f->y0; d.z0 = (Real)f->z0;
  return d;
}

template <class Real> Tables<Real> tables_of(const qed_ctx *c);
template <> inline Tables<float> tables_of<float>(const qed_ctx *c) {
  return Tables<float>{c->R32, c->F32, c->Y32, c->P32, c->Yp32, to_r<float>(c->gl),
                       to_r<float>(c->gy), to_r<float>(c->gk), to_r<float>(c->glp),
                       to_r<float>(c->gkp)};
}
template <> inline Tables<double> tables_of<double>(const qed_ctx *c) {
  return Tables<double>{c->R64, c->F64, c->Y64, c->P64, c->Yp64, to_r<double>(c->gl),
                        to_r<double>(c->gy), to_r<double>(c->gk), to_r<double>(c->glp),
                        to_r<double>(c->gkp)};
}

Consts consts_of(const qed_ctx *c);
Out out_of(const qed_ctx *c);

}  // namespace qed
