// qed_pic.cu -- the particle-in-cell loop around the QED step: current
// deposition, the Yee field update and the node grid the particle gather
// reads (qed_pic_deposit, qed_pic_fields, qed_pic_step).
//
// The paper adds its QED module to a PIC code (introduction) whose field
// solver it does not describe; this is the standard explicit scheme.  Fields
// live on Yee's staggered grid in float, [nz][ny][nx] per component (x
// fastest), periodic:
//   ex, jx at (i+1/2, j, k)     bx at (i, j+1/2, k+1/2)
//   ey, jy at (i, j+1/2, k)     by at (i+1/2, j, k+1/2)
//   ez, jz at (i, j, k+1/2)     bz at (i+1/2, j+1/2, k)
// and are advanced by the leapfrog of dB/dt = -curl E, dE/dt = curl B - J in
// the units of the library (J in e n_c c).
//
// Kernels.  The field kernels are stencils bound by HBM bandwidth: one thread
// per cell, a CTA per run of 128 cells along x (coalesced), the y/z
// neighbours coming from planes that L2 still holds.  One step is four
// passes -- B half-step, E step (which zeroes J behind it), B half-step, node
// grid -- because each needs its neighbours' results of the one before.  The
// deposit is one thread per particle, grid-stride over a persistent grid:
// 8 CIC weights x 3 components at their staggered positions, reduced in L2
// by atomics -- the two x-neighbours of each stencil row by one 16-byte
// vector atomic where they share an aligned group of four floats (3 rows
// in 4), so about 15 atomic operations per particle instead of 24.
#include <cmath>
#include <cstdio>

#include "qed_internal.h"

namespace qed {
namespace {

int cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return QED_OK;
  fprintf(stderr, "libqed: %s: %s\n", what, cudaGetErrorString(e));
  return QED_ERR_CUDA;
}

constexpr int FIELD_THREADS = 128;
constexpr int DEPOSIT_THREADS = 256;

struct YeeArgs {
  float *ex, *ey, *ez, *bx, *by, *bz, *jx, *jy, *jz;
  float4 *nodes;
  int nx, ny, nz;
  float idx, idy, idz;  // inverse spacings
};

YeeArgs yee_args(const qed_yee *y) {
  YeeArgs a;
  a.ex = y->ex; a.ey = y->ey; a.ez = y->ez;
  a.bx = y->bx; a.by = y->by; a.bz = y->bz;
  a.jx = y->jx; a.jy = y->jy; a.jz = y->jz;
  a.nodes = reinterpret_cast<float4 *>(y->nodes);
  a.nx = y->nx; a.ny = y->ny; a.nz = y->nz;
  a.idx = (float)(1.0 / y->dx); a.idy = (float)(1.0 / y->dy); a.idz = (float)(1.0 / y->dz);
  return a;
}

// The cell of this thread and its periodic neighbours: c = cell (i, j, k),
// xp/xm = (i +- 1, j, k), yp/ym, zp/zm likewise.  Rows (j, k) run along
// blockIdx.x, runs of x along blockIdx.y.
struct Cell {
  int64_t c, xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ bool cell_of(const YeeArgs &A, Cell &q) {
  const int i = blockIdx.y * FIELD_THREADS + threadIdx.x;
  if (i >= A.nx) return false;
  const int row = blockIdx.x, j = row % A.ny, k = row / A.ny;
  const int64_t nx = A.nx, plane = (int64_t)A.nx * A.ny;
  const int ip = i + 1 == A.nx ? 0 : i + 1, im = i == 0 ? A.nx - 1 : i - 1;
  const int jp = j + 1 == A.ny ? 0 : j + 1, jm = j == 0 ? A.ny - 1 : j - 1;
  const int kp = k + 1 == A.nz ? 0 : k + 1, km = k == 0 ? A.nz - 1 : k - 1;
  const int64_t base = (int64_t)k * plane + (int64_t)j * nx;
  q.c = base + i;
  q.xp = base + ip;
  q.xm = base + im;
  q.yp = (int64_t)k * plane + (int64_t)jp * nx + i;
  q.ym = (int64_t)k * plane + (int64_t)jm * nx + i;
  q.zp = (int64_t)kp * plane + (int64_t)j * nx + i;
  q.zm = (int64_t)km * plane + (int64_t)j * nx + i;
  return true;
}

// B -= h curl E at the B positions (forward differences of E).
__global__ void __launch_bounds__(FIELD_THREADS) k_yee_b_half(YeeArgs A, float h) {
  Cell q;
  if (!cell_of(A, q)) return;
  const float ex = A.ex[q.c], ey = A.ey[q.c], ez = A.ez[q.c];
  const float cx = (A.ez[q.yp] - ez) * A.idy - (A.ey[q.zp] - ey) * A.idz;
  const float cy = (A.ex[q.zp] - ex) * A.idz - (A.ez[q.xp] - ez) * A.idx;
  const float cz = (A.ey[q.xp] - ey) * A.idx - (A.ex[q.yp] - ex) * A.idy;
  A.bx[q.c] -= h * cx;
  A.by[q.c] -= h * cy;
  A.bz[q.c] -= h * cz;
}

// E += dt (curl B - J) at the E positions (backward differences of B); J is
// zeroed for the next deposit.
__global__ void __launch_bounds__(FIELD_THREADS) k_yee_e(YeeArgs A, float dt) {
  Cell q;
  if (!cell_of(A, q)) return;
  const float bx = A.bx[q.c], by = A.by[q.c], bz = A.bz[q.c];
  const float cx = (bz - A.bz[q.ym]) * A.idy - (by - A.by[q.zm]) * A.idz;
  const float cy = (bx - A.bx[q.zm]) * A.idz - (bz - A.bz[q.xm]) * A.idx;
  const float cz = (by - A.by[q.xm]) * A.idx - (bx - A.bx[q.ym]) * A.idy;
  A.ex[q.c] += dt * (cx - A.jx[q.c]);
  A.ey[q.c] += dt * (cy - A.jy[q.c]);
  A.ez[q.c] += dt * (cz - A.jz[q.c]);
  A.jx[q.c] = 0.f;
  A.jy[q.c] = 0.f;
  A.jz[q.c] = 0.f;
}

// Node (i, j, k): E components the mean of their two staggered neighbours
// along their own axis, B components the mean of their four neighbours in
// the plane normal to them.
__global__ void __launch_bounds__(FIELD_THREADS) k_yee_nodes(YeeArgs A) {
  Cell q;
  if (!cell_of(A, q)) return;
  // the diagonal neighbours (j-1, k-1), (i-1, k-1), (i-1, j-1): the index is
  // linear in each of i, j, k, so their offsets add
  const int64_t ym_zm = q.ym - q.c + q.zm, xm_zm = q.xm - q.c + q.zm, xm_ym = q.xm - q.c + q.ym;
  float4 a, b;
  a.x = 0.5f * (A.ex[q.c] + A.ex[q.xm]);
  a.y = 0.5f * (A.ey[q.c] + A.ey[q.ym]);
  a.z = 0.5f * (A.ez[q.c] + A.ez[q.zm]);
  a.w = 0.25f * (A.bx[q.c] + A.bx[q.ym] + A.bx[q.zm] + A.bx[ym_zm]);
  b.x = 0.25f * (A.by[q.c] + A.by[q.xm] + A.by[q.zm] + A.by[xm_zm]);
  b.y = 0.25f * (A.bz[q.c] + A.bz[q.xm] + A.bz[q.ym] + A.bz[xm_ym]);
  b.z = 0.f;
  b.w = 0.f;
  A.nodes[2 * q.c] = a;
  A.nodes[2 * q.c + 1] = b;
}

template <class Real> struct DepArgs {
  const Real *x, *y, *z, *px, *py, *pz, *w;
  const int64_t *d_n, *d_lim;
  int64_t cap;
  float *jx, *jy, *jz;
  int nx, ny, nz;
  Real idx, idy, idz, x0, y0, z0;
  Real scale;   // q weight_unit / (dx dy dz)
  Real half_dt;
  qed_counters *cnt;
};

// The two x-neighbours a0, a1 of one row of the stencil: one 16-byte vector
// atomic (the other two lanes add zero) when both lie in one aligned group of
// four floats inside the array, else a scalar atomic each (a row wrapping
// around the periodic boundary, a pair across a group, or nx = 1, where
// a1 == a0).
__device__ __forceinline__ void add_pair(float *J, int64_t ncell, int64_t a0, int64_t a1, float v0,
                                         float v1) {
  const int64_t g = a0 & ~(int64_t)3;
  const int l = (int)(a0 & 3);
  if (a1 == a0 + 1 && l != 3 && g + 3 < ncell) {
    const float4 v = l == 0 ? make_float4(v0, v1, 0.f, 0.f)
                   : l == 1 ? make_float4(0.f, v0, v1, 0.f)
                            : make_float4(0.f, 0.f, v0, v1);
    atomicAdd(reinterpret_cast<float4 *>(J + g), v);
  } else {
    atomicAdd(J + a0, v0);
    atomicAdd(J + a1, v1);
  }
}

// CIC spread of `amount` at reduced coordinates (fx, fy, fz) (cells from the
// origin of the component's staggered lattice).
template <class Real>
__device__ __forceinline__ void spread(float *J, const DepArgs<Real> &A, Real fx, Real fy, Real fz,
                                       Real amount) {
  const Real ix = floor(fx), iy = floor(fy), iz = floor(fz);
  const Real wx = fx - ix, wy = fy - iy, wz = fz - iz;
  int64_t i0 = (int64_t)ix % A.nx, j0 = (int64_t)iy % A.ny, k0 = (int64_t)iz % A.nz;
  if (i0 < 0) i0 += A.nx;
  if (j0 < 0) j0 += A.ny;
  if (k0 < 0) k0 += A.nz;
  const int64_t i1 = i0 + 1 == A.nx ? 0 : i0 + 1;
  const int64_t j1 = j0 + 1 == A.ny ? 0 : j0 + 1;
  const int64_t k1 = k0 + 1 == A.nz ? 0 : k0 + 1;
  const int64_t nx = A.nx, plane = (int64_t)A.nx * A.ny, ncell = plane * A.nz;
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj) {
      const Real wr = amount * (dj ? wy : (Real)1 - wy) * (dk ? wz : (Real)1 - wz);
      const int64_t row = (dk ? k1 : k0) * plane + (dj ? j1 : j0) * nx;
      add_pair(J, ncell, row + i0, row + i1, (float)(wr * ((Real)1 - wx)), (float)(wr * wx));
    }
}

template <class Real>
__global__ void __launch_bounds__(DEPOSIT_THREADS) k_pic_deposit(DepArgs<Real> A) {
  int64_t n = *A.d_n;
  if (A.d_lim && *A.d_lim < n) n = *A.d_lim;
  if (n > A.cap) n = A.cap;
  const Real lim = (Real)4.0e15;  // reduced coordinates beyond this are not finite cells
  unsigned bad = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const Real px = A.px[p], py = A.py[p], pz = A.pz[p];
    const Real ig = (Real)1 / sqrt((Real)1 + px * px + py * py + pz * pz);
    const Real vx = px * ig, vy = py * ig, vz = pz * ig;
    const Real fx = (A.x[p] - A.half_dt * vx - A.x0) * A.idx;
    const Real fy = (A.y[p] - A.half_dt * vy - A.y0) * A.idy;
    const Real fz = (A.z[p] - A.half_dt * vz - A.z0) * A.idz;
    if (!(fabs(fx) < lim && fabs(fy) < lim && fabs(fz) < lim)) {  // also false for NaN
      bad = 1;
      continue;
    }
    const Real a = A.scale * A.w[p];
    spread(A.jx, A, fx - (Real)0.5, fy, fz, a * vx);
    spread(A.jy, A, fx, fy - (Real)0.5, fz, a * vy);
    spread(A.jz, A, fx, fy, fz - (Real)0.5, a * vz);
  }
  if (bad) atomicOr(&A.cnt->status, (unsigned)QED_STATUS_NONFINITE);
}

bool yee_ok(const qed_yee *y) {
  if (!y || y->nx < 1 || y->ny < 1 || y->nz < 1 || y->nx > 65536 || y->ny > 65536 ||
      y->nz > 65536 || (int64_t)y->ny * y->nz > 0x7fffffffLL)
    return false;
  if (!(y->dx > 0) || !(y->dy > 0) || !(y->dz > 0) || !std::isfinite(y->dx) ||
      !std::isfinite(y->dy) || !std::isfinite(y->dz) || !std::isfinite(y->x0) ||
      !std::isfinite(y->y0) || !std::isfinite(y->z0))
    return false;
  const void *p[] = {y->ex, y->ey, y->ez, y->bx, y->by, y->bz, y->jx, y->jy, y->jz, y->nodes};
  for (const void *q : p)
    if (!q || (reinterpret_cast<uintptr_t>(q) & 15) != 0) return false;
  return true;
}

bool courant_ok(const qed_yee *y, double dt) {
  double s = 0;
  if (y->nx > 1) s += 1.0 / (y->dx * y->dx);
  if (y->ny > 1) s += 1.0 / (y->dy * y->dy);
  if (y->nz > 1) s += 1.0 / (y->dz * y->dz);
  return dt * std::sqrt(s) < 1.0;
}

cudaError_t launch_fields(qed_ctx *c, const qed_yee *y, bool advance, cudaStream_t st) {
  const YeeArgs A = yee_args(y);
  const dim3 grid((unsigned)((int64_t)y->ny * y->nz), (unsigned)((y->nx + FIELD_THREADS - 1) / FIELD_THREADS));
  const float dt = (float)c->cfg.dt;
  if (advance) {
    k_yee_b_half<<<grid, FIELD_THREADS, 0, st>>>(A, 0.5f * dt);
    k_yee_e<<<grid, FIELD_THREADS, 0, st>>>(A, dt);
    k_yee_b_half<<<grid, FIELD_THREADS, 0, st>>>(A, 0.5f * dt);
    c->launches += 3;
  }
  k_yee_nodes<<<grid, FIELD_THREADS, 0, st>>>(A);
  c->launches += 1;
  return cudaGetLastError();
}

template <class Real>
cudaError_t launch_deposit(qed_ctx *c, const qed_species *s, const qed_yee *y, double weight_unit,
                           const int64_t *d_lim, cudaStream_t st) {
  DepArgs<Real> A;
  A.x = static_cast<const Real *>(s->x); A.y = static_cast<const Real *>(s->y);
  A.z = static_cast<const Real *>(s->z);
  A.px = static_cast<const Real *>(s->px); A.py = static_cast<const Real *>(s->py);
  A.pz = static_cast<const Real *>(s->pz); A.w = static_cast<const Real *>(s->w);
  A.d_n = s->d_n; A.d_lim = d_lim; A.cap = s->capacity;
  A.jx = y->jx; A.jy = y->jy; A.jz = y->jz;
  A.nx = y->nx; A.ny = y->ny; A.nz = y->nz;
  A.idx = (Real)(1.0 / y->dx); A.idy = (Real)(1.0 / y->dy); A.idz = (Real)(1.0 / y->dz);
  A.x0 = (Real)y->x0; A.y0 = (Real)y->y0; A.z0 = (Real)y->z0;
  A.scale = (Real)((double)s->q * weight_unit / (y->dx * y->dy * y->dz));
  A.half_dt = (Real)(0.5 * c->cfg.dt);
  A.cnt = c->d_counters;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pic_deposit<Real>,
                                                                DEPOSIT_THREADS, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  // no more CTAs than the capacity needs
  const int64_t need = (s->capacity + DEPOSIT_THREADS - 1) / DEPOSIT_THREADS;
  int64_t blocks = (int64_t)c->num_sms * per_sm;
  if (need < blocks) blocks = need;
  if (blocks < 1) blocks = 1;
  k_pic_deposit<Real><<<(unsigned)blocks, DEPOSIT_THREADS, 0, st>>>(A);
  c->launches += 1;
  return cudaGetLastError();
}

__global__ void k_copy_counts(int64_t *dst, const int64_t *a, const int64_t *b) {
  dst[0] = *a;
  dst[1] = *b;
}

// a lepton species (an empty one of any charge is accepted: it deposits nothing)
bool lepton_ok(const qed_species *s) {
  if (!s || !s->d_n || s->capacity < 0) return false;
  if (s->capacity == 0) return true;
  return s->q != 0 && s->x && s->y && s->z && s->px && s->py && s->pz && s->w;
}

}  // namespace
}  // namespace qed

using namespace qed;

extern "C" int qed_pic_deposit(qed_ctx *c, const qed_species *s, const qed_yee *y,
                               double weight_unit, const int64_t *d_count, qed_stream_t stream) {
  if (!c || !lepton_ok(s) || !yee_ok(y) || !std::isfinite(weight_unit)) return QED_ERR_ARG;
  if (s->capacity == 0) return QED_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = c->cfg.precision == QED_FP64
                      ? launch_deposit<double>(c, s, y, weight_unit, d_count, st)
                      : launch_deposit<float>(c, s, y, weight_unit, d_count, st);
  return cuda_fail(e, "qed_pic_deposit");
}

extern "C" int qed_pic_fields(qed_ctx *c, const qed_yee *y, int advance, qed_stream_t stream) {
  if (!c || !yee_ok(y) || (advance && !courant_ok(y, c->cfg.dt))) return QED_ERR_ARG;
  return cuda_fail(launch_fields(c, y, advance != 0, (cudaStream_t)stream), "qed_pic_fields");
}

extern "C" int qed_pic_step(qed_ctx *c, const qed_species *e, const qed_species *p,
                            const qed_species *g, const qed_yee *y, double weight_unit, int64_t step,
                            qed_stream_t stream) {
  if (!c || !yee_ok(y) || !courant_ok(y, c->cfg.dt) || !std::isfinite(weight_unit) ||
      !lepton_ok(e) || !lepton_ok(p))
    return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // lepton counts before the step: the leptons its pairs create are
  // deposited from the next step on
  k_copy_counts<<<1, 1, 0, st>>>(c->pic_n, e->d_n, p->d_n);
  c->launches += 1;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "qed_pic_step");
  qed_fields f{};
  f.mode = QED_FIELDS_GRID;
  f.nx = y->nx; f.ny = y->ny; f.nz = y->nz;
  f.grid = y->nodes;
  f.dx = y->dx; f.dy = y->dy; f.dz = y->dz;
  f.x0 = y->x0; f.y0 = y->y0; f.z0 = y->z0;
  int rc = qed_step_fused(c, e, p, g, &f, step, stream);
  if (rc == QED_OK) rc = qed_pic_deposit(c, e, y, weight_unit, c->pic_n, stream);
  if (rc == QED_OK) rc = qed_pic_deposit(c, p, y, weight_unit, c->pic_n + 1, stream);
  if (rc == QED_OK) rc = qed_pic_fields(c, y, 1, stream);
  return rc;
}
