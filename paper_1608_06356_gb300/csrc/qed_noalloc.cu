// qed_noalloc.cu -- qed_compact_noalloc: stable in-place removal of dead
// particles that allocates no memory at all.
//
// Why it exists: some callers cannot allocate device memory when they call
// us -- a host application that owns every device allocation through its own
// pool or arena, a plugin sandbox that forbids cudaMalloc, or code running
// where an allocation would synchronise the device.  qed_compact needs a
// qed_ctx, and creating one allocates tables and scan state.  This variant
// keeps its only scratch -- the look-back state of the single-pass scan and
// two counters -- in a file-scope static __device__ array instead, so a
// caller passes the particle buffers (inputs and outputs) and nothing else.
//
// Limits and sharing:
//   * at most NOALLOC_MAX_PARTICLES (2^24 = 16,777,216) particles per species
//     (the capacity is checked; larger calls return QED_ERR_CAPACITY);
//   * the array (512 KiB + 64 B) exists once per device that loads the
//     library and is held until the process exits;
//   * every call uses the same array, which keeps the previous call's
//     contents.  Stale scan words are made invalid by an epoch that advances
//     with every call, and the two counters that must start at zero are
//     cleared (cudaMemsetAsync on the stream) before every launch;
//   * calls that overlap on the GPU (on different streams without ordering,
//     or from different threads at once) race on the array: issue them to one
//     stream or order them;
//   * a count *d_n above the capacity is clamped to the capacity (and
//     QED_STATUS_CAPACITY is reported), so no tile reaches past the array.
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (once per device, with that device current); make that
// first call before any stream capture.
#include <cstdio>
#include <mutex>

#include "qed_device.cuh"
#include "qed_internal.h"

namespace qed {
namespace {

constexpr int64_t NOALLOC_MAX_PARTICLES = (int64_t)1 << 24;
constexpr int64_t NOALLOC_MAX_TILES = NOALLOC_MAX_PARTICLES / TILE;
// [0, NOALLOC_MAX_TILES): look-back state words; then 8 words of counters
// (viewed as unsigned int: [0] tile counter, [1] done counter, [2] epoch).
constexpr int64_t NOALLOC_WORDS = NOALLOC_MAX_TILES + 8;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_WORDS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned long long *g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Device address of the static array on the current device (looked up once).
int scratch_for_current_device(unsigned long long **ptr, int *num_sms) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    fprintf(stderr, "libqed: qed_compact_noalloc: no usable current device\n");
    return QED_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "libqed: qed_compact_noalloc: cudaGetSymbolAddress failed: %s\n",
              cudaGetErrorString(e));
      return QED_ERR_CUDA;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) {
      fprintf(stderr, "libqed: qed_compact_noalloc: device query failed\n");
      return QED_ERR_CUDA;
    }
    g_num_sms[dev] = sms;
    g_scratch_ptr[dev] = static_cast<unsigned long long *>(p);
  }
  *ptr = g_scratch_ptr[dev];
  *num_sms = g_num_sms[dev];
  return QED_OK;
}

template <class Real> struct NoallocCompactArgs {
  Real *v[13];  // x y z px py pz w ex ey ez bx by bz (field arrays may be null)
  uint64_t *id;
  uint8_t *alive;
  uint32_t *tag;       // optional
  int64_t *d_n;
  int64_t capacity;    // the species' capacity (<= NOALLOC_MAX_PARTICLES)
  uint32_t *d_status;  // caller-owned, may be null
  ScanState scan;
};

// Same algorithm as the context-based compaction: every tile loads its
// particles into registers before publishing its count, and writes only after
// all earlier tiles have published, so the in-place move never overwrites
// unread data.
template <class Real>
__global__ void __launch_bounds__(TILE) k_compact_noalloc(NoallocCompactArgs<Real> A) {
  __shared__ uint32_t scan_sm[33];
  __shared__ long long s_meta[5];
  if (threadIdx.x == 0) {
    s_meta[2] = *(volatile int64_t *)A.d_n;
    s_meta[3] = (long long)A.scan.sync[2];
  }
  __syncthreads();
  // a count above the capacity (a caller's error) is clamped to it, so the
  // tiles stay inside the static scan state and the caller's arrays
  const int64_t n_in = s_meta[2];
  const int64_t n = n_in < 0 ? 0 : (n_in > A.capacity ? A.capacity : n_in);
  const uint32_t epoch = (uint32_t)s_meta[3];
  const int64_t ntiles = (n + TILE - 1) / TILE;
  const bool fields = A.v[7] != nullptr;
  uint32_t status = n != n_in ? (uint32_t)QED_STATUS_CAPACITY : 0u;
  for (;;) {
    if (threadIdx.x == 0) s_meta[0] = (long long)atomicAdd(&A.scan.sync[0], 1u);
    __syncthreads();
    const int64_t t = s_meta[0];
    __syncthreads();
    if (t >= ntiles || t >= A.scan.max_tiles) break;
    const int64_t i = t * TILE + threadIdx.x;
    uint32_t keep = 0;
    Real r[13];
    uint64_t id = 0;
    uint32_t tg = 0;
    if (i < n && A.alive[i]) {
      keep = 1;
      if (A.tag) tg = A.tag[i];
#pragma unroll
      for (int c = 0; c < 7; ++c) r[c] = A.v[c][i];
      if (fields) {
#pragma unroll
        for (int c = 7; c < 13; ++c) r[c] = A.v[c][i];
      }
      id = A.id[i];
    }
    uint32_t excl = block_excl_scan(keep, scan_sm);
    uint32_t agg = scan_sm[32];
    if (threadIdx.x < 32) {
      uint32_t st_tile = 0;
      uint32_t pre = lookback_warp(A.scan, t, epoch, agg, st_tile);
      // any lane of the walk may have given up (warp 0 runs converged here)
      const bool gave_up = __any_sync(0xFFFFFFFFu, (st_tile & QED_STATUS_TIMEOUT) != 0);
      status |= st_tile;
      if (threadIdx.x == 0) {
        s_meta[1] = pre;
        // no valid prefix after a look-back that gave up: write nothing (see
        // the context-based compaction); the status word reports it
        s_meta[4] = gave_up ? 1 : 0;
        if (t == ntiles - 1 && !s_meta[4]) *A.d_n = (int64_t)pre + agg;
      }
    }
    __syncthreads();
    if (keep && !s_meta[4]) {
      const int64_t d = s_meta[1] + excl;
#pragma unroll
      for (int c = 0; c < 7; ++c) A.v[c][d] = r[c];
      if (fields) {
#pragma unroll
        for (int c = 7; c < 13; ++c) A.v[c][d] = r[c];
      }
      A.id[d] = id;
      A.alive[d] = 1;
      if (A.tag) A.tag[d] = tg;
    }
  }
  if (threadIdx.x == 0 && status && A.d_status) atomicOr(A.d_status, status);
  // the last CTA to finish resets the tile counter and advances the epoch
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(&A.scan.sync[1], 1u);
    if (prev == gridDim.x - 1) {
      A.scan.sync[0] = 0u;
      A.scan.sync[1] = 0u;
      A.scan.sync[2] = epoch + 1u;
      __threadfence();
    }
  }
}

template <class Real>
int launch_noalloc(const qed_species *s, uint32_t *d_status, cudaStream_t st) {
  unsigned long long *scratch = nullptr;
  int sms = 0;
  int rc = scratch_for_current_device(&scratch, &sms);
  if (rc != QED_OK) return rc;
  unsigned int *sync = reinterpret_cast<unsigned int *>(scratch + NOALLOC_MAX_TILES);
  // tile and done counters must start at zero; the epoch (sync[2]) is kept
  cudaError_t e = cudaMemsetAsync(sync, 0, 2 * sizeof(unsigned int), st);
  if (e != cudaSuccess) {
    fprintf(stderr, "libqed: qed_compact_noalloc: %s\n", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  NoallocCompactArgs<Real> a{};
  void *arrs[13] = {s->x, s->y, s->z, s->px, s->py, s->pz, s->w,
                    s->ex, s->ey, s->ez, s->bx, s->by, s->bz};
  for (int c = 0; c < 13; ++c) a.v[c] = static_cast<Real *>(arrs[c]);
  a.id = s->id;
  a.alive = s->alive;
  a.tag = s->tag;
  a.d_n = s->d_n;
  a.capacity = s->capacity;
  a.d_status = d_status;
  a.scan = ScanState{scratch, sync, NOALLOC_MAX_TILES};
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_compact_noalloc<Real>, TILE, 0);
  if (e != cudaSuccess) {
    fprintf(stderr, "libqed: qed_compact_noalloc: %s\n", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  if (per_sm < 1) per_sm = 1;
  k_compact_noalloc<Real><<<sms * per_sm, TILE, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "libqed: qed_compact_noalloc: %s\n", cudaGetErrorString(e));
    return QED_ERR_CUDA;
  }
  return QED_OK;
}

}  // namespace
}  // namespace qed

extern "C" int qed_compact_noalloc(const qed_species *s, int precision, uint32_t *d_status,
                                   qed_stream_t stream) {
  using namespace qed;
  if (!s || (precision != QED_FP32 && precision != QED_FP64) || !s->d_n || s->capacity < 0)
    return QED_ERR_ARG;
  if (s->capacity > NOALLOC_MAX_PARTICLES) {
    fprintf(stderr,
            "libqed: qed_compact_noalloc: capacity %lld exceeds the static scratch limit of "
            "%lld particles\n",
            (long long)s->capacity, (long long)NOALLOC_MAX_PARTICLES);
    return QED_ERR_CAPACITY;
  }
  if (s->capacity > 0 && (!s->x || !s->y || !s->z || !s->px || !s->py || !s->pz || !s->w ||
                          !s->id || !s->alive))
    return QED_ERR_ARG;
  const bool any_f = s->ex || s->ey || s->ez || s->bx || s->by || s->bz;
  const bool all_f = s->ex && s->ey && s->ez && s->bx && s->by && s->bz;
  if (any_f && !all_f) return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == QED_FP64 ? launch_noalloc<double>(s, d_status, st)
                               : launch_noalloc<float>(s, d_status, st);
}
