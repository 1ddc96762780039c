// qed_host.cu -- the lepton stage of the QED step for leptons held in host
// memory: the ensemble is streamed through the GPU in chunks, with the copies
// of one chunk overlapping the step of another.
//
// Three device staging buffers of `chunk` leptons rotate through three
// streams: chunk k is copied in on the input stream (once its buffer's
// previous chunk has been copied out), stepped on the caller's stream -- the
// same launches as qed_step_fused's lepton stage, appending photons to the
// device photon species -- and its positions and momenta copied back on the
// output stream.  The photons a chunk appended go to the host mirror of the
// photon species on the output stream too: by a copy kernel that reads the
// chunk's range on the device and writes through host-mapped pointers, so
// that every chunk is queued at once and the host waits only at the end (or,
// for mirror memory the device cannot map, by copies whose ranges the host
// reads after each chunk).  Particle ids key the random
// streams, so chunking changes no result, only the order of the photons
// (chunks in order; within a chunk as the lepton step appends them).
#include <cstdio>
#include <cstring>

#include "qed_internal.h"

namespace qed {
template <class Real>
cudaError_t launch_lepton(qed_ctx *, const qed_species *, const qed_species *, const qed_species *,
                          const qed_fields *, int64_t, int, cudaStream_t);

namespace {

constexpr int MODE_FUSED_ = 2;  // gather, push and emission (the lepton stage of qed_step_fused)

int cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return QED_OK;
  fprintf(stderr, "libqed: %s: %s\n", what, cudaGetErrorString(e));
  return QED_ERR_CUDA;
}

__global__ void k_set_count(int64_t *d_n, int64_t v) { *d_n = v; }
__global__ void k_mark_count(int64_t *dst, const int64_t *src) { *dst = *src; }

// Copy of the photons appended by one chunk, [*lo, *hi) clamped to the
// capacity, from the device photon species to its host mirror through
// host-mapped pointers: the range is read on the device, so no host round
// trip is needed between the chunks.
constexpr int MAX_PARRAYS = 16;
struct PhotonCopy {
  const char *src[MAX_PARRAYS];
  char *dst[MAX_PARRAYS];
  int esz[MAX_PARRAYS];
  int wide[MAX_PARRAYS];  // 16: both bases 16-byte aligned; 4: 4-byte aligned; else bytes
  int np;
  const int64_t *lo, *hi;
  int64_t cap;
};

__global__ void __launch_bounds__(256) k_copy_photons(PhotonCopy A) {
  int64_t lo = *A.lo, hi = *A.hi;
  lo = lo < A.cap ? lo : A.cap;
  hi = hi < A.cap ? hi : A.cap;
  if (hi <= lo) return;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (int a = 0; a < A.np; ++a) {
    const int64_t b0 = lo * A.esz[a], b1 = hi * A.esz[a];
    if (A.esz[a] % 4 || A.wide[a] < 4) {  // bytes (alive flags, or unaligned bases)
      for (int64_t q = b0 + t0; q < b1; q += nt) A.dst[a][q] = A.src[a][q];
      continue;
    }
    // 4-byte words up to a 16-byte boundary, 16-byte words, 4-byte words after
    const int64_t m0 = (b0 + 15) & ~(int64_t)15, m1 = b1 & ~(int64_t)15;
    if (m0 >= m1 || A.wide[a] < 16) {
      for (int64_t q = b0 / 4 + t0; q < b1 / 4; q += nt)
        reinterpret_cast<uint32_t *>(A.dst[a])[q] = reinterpret_cast<const uint32_t *>(A.src[a])[q];
      continue;
    }
    for (int64_t q = b0 / 4 + t0; q < m0 / 4; q += nt)
      reinterpret_cast<uint32_t *>(A.dst[a])[q] = reinterpret_cast<const uint32_t *>(A.src[a])[q];
    for (int64_t q = m0 / 16 + t0; q < m1 / 16; q += nt)
      reinterpret_cast<uint4 *>(A.dst[a])[q] = reinterpret_cast<const uint4 *>(A.src[a])[q];
    for (int64_t q = m1 / 4 + t0; q < b1 / 4; q += nt)
      reinterpret_cast<uint32_t *>(A.dst[a])[q] = reinterpret_cast<const uint32_t *>(A.src[a])[q];
  }
}

// One array of the lepton species as the host step moves it: host pointer,
// bytes per element, device staging offset, and whether it is copied back.
struct Lane {
  char *host;
  size_t esz;
  size_t off;
  bool back;
};

constexpr int NBUF = 3;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// The arrays of a lepton species, in staging order; *per_buf = staging bytes
// of one buffer for `chunk` leptons.
int lanes_of(const qed_species *s, size_t real, int64_t chunk, Lane out[16], size_t *per_buf) {
  int n = 0;
  size_t off = 0;
  auto add = [&](void *p, size_t esz, bool back) {
    out[n++] = Lane{static_cast<char *>(p), esz, off, back};
    off += align256(esz * (size_t)chunk);
  };
  void *state[6] = {s->x, s->y, s->z, s->px, s->py, s->pz};
  for (void *p : state) add(p, real, true);
  add(s->w, real, false);
  add(s->id, sizeof(uint64_t), false);
  void *fld[6] = {s->ex, s->ey, s->ez, s->bx, s->by, s->bz};
  if (s->ex)
    for (void *p : fld) add(p, real, false);
  if (s->od_p) {
    add(s->od_p, real, true);
    add(s->od_r, real, true);
  }
  if (s->tag) add(s->tag, sizeof(uint32_t), false);
  *per_buf = off;
  return n;
}

// The device species of staging buffer b.
qed_species staging_species(qed_ctx *c, const qed_species *h, const Lane *L, int nl, int b,
                            int64_t chunk) {
  char *base = static_cast<char *>(c->hs_mem) + (size_t)b * c->hs_per_buf;
  qed_species s{};
  void **dst[6] = {&s.x, &s.y, &s.z, &s.px, &s.py, &s.pz};
  int k = 0;
  for (int i = 0; i < 6; ++i) *dst[i] = base + L[k++].off;
  s.w = base + L[k++].off;
  s.id = reinterpret_cast<uint64_t *>(base + L[k++].off);
  if (h->ex) {
    void **fd[6] = {&s.ex, &s.ey, &s.ez, &s.bx, &s.by, &s.bz};
    for (int i = 0; i < 6; ++i) *fd[i] = base + L[k++].off;
  }
  if (h->od_p) {
    s.od_p = base + L[k++].off;
    s.od_r = base + L[k++].off;
  }
  if (h->tag) s.tag = reinterpret_cast<uint32_t *>(base + L[k++].off);
  (void)nl;
  s.d_n = c->hs_dn + b;
  s.capacity = chunk;
  s.q = h->q;
  return s;
}

// The arrays of a photon species and of its host mirror (the mirror must have
// every array the device species has).
int photon_arrays(const qed_species *g, const qed_species *gh, size_t real, void *dev[16],
                  void *host[16], size_t esz[16]) {
  int n = 0;
  auto add = [&](void *d, void *h, size_t e) {
    if (!d) return true;
    if (!h) return false;
    dev[n] = d; host[n] = h; esz[n] = e; ++n;
    return true;
  };
  bool ok = add(g->x, gh->x, real) && add(g->y, gh->y, real) && add(g->z, gh->z, real) &&
            add(g->px, gh->px, real) && add(g->py, gh->py, real) && add(g->pz, gh->pz, real) &&
            add(g->w, gh->w, real) && add(g->id, gh->id, sizeof(uint64_t)) &&
            add(g->alive, gh->alive, 1) && add(g->ex, gh->ex, real) && add(g->ey, gh->ey, real) &&
            add(g->ez, gh->ez, real) && add(g->bx, gh->bx, real) && add(g->by, gh->by, real) &&
            add(g->bz, gh->bz, real) && add(g->tag, gh->tag, sizeof(uint32_t));
  return ok ? n : -1;
}

int ensure_host_step(qed_ctx *c, size_t per_buf) {
  if (!c->hs_in) {
    if (cudaStreamCreateWithFlags(&c->hs_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->hs_out, cudaStreamNonBlocking) != cudaSuccess)
      return QED_ERR_CUDA;
    for (int i = 0; i < 3 * NBUF; ++i)
      if (cudaEventCreateWithFlags(&c->hs_ev[i], cudaEventDisableTiming) != cudaSuccess)
        return QED_ERR_CUDA;
    if (cudaMalloc(&c->hs_dn, (2 * NBUF + 1) * sizeof(int64_t)) != cudaSuccess) return QED_ERR_NOMEM;
    if (cudaHostAlloc(reinterpret_cast<void **>(&c->hs_cnt), 2 * NBUF * sizeof(int64_t),
                      cudaHostAllocDefault) != cudaSuccess)
      return QED_ERR_NOMEM;
  }
  if (per_buf > c->hs_per_buf) {
    if (c->hs_mem) {
      cudaFree(c->hs_mem);
      c->hs_mem = nullptr;
      c->hs_per_buf = 0;
    }
    if (cudaMalloc(&c->hs_mem, NBUF * per_buf) != cudaSuccess) return QED_ERR_NOMEM;
    c->hs_per_buf = per_buf;
  }
  return QED_OK;
}

}  // namespace

void free_host_step(qed_ctx *c) {
  if (c->hs_mem) cudaFree(c->hs_mem);
  if (c->hs_dn) cudaFree(c->hs_dn);
  if (c->hs_cnt) cudaFreeHost(c->hs_cnt);
  for (int i = 0; i < 3 * NBUF; ++i)
    if (c->hs_ev[i]) cudaEventDestroy(c->hs_ev[i]);
  if (c->hs_in) cudaStreamDestroy(c->hs_in);
  if (c->hs_out) cudaStreamDestroy(c->hs_out);
}

int lepton_step_host(qed_ctx *c, const qed_species *lh, const qed_species *g,
                     const qed_species *gh, const qed_fields *f, int64_t step, int64_t chunk,
                     cudaStream_t st) {
  const bool f64 = c->cfg.precision == QED_FP64;
  const size_t real = f64 ? sizeof(double) : sizeof(float);
  const int64_t n = *lh->d_n;
  if (n < 0 || n > lh->capacity) return QED_ERR_ARG;
  Lane L[16];
  size_t per_buf = 0;
  const int nl = lanes_of(lh, real, chunk, L, &per_buf);
  void *pdev[16], *phost[16];
  size_t pesz[16];
  const int np = gh ? photon_arrays(g, gh, real, pdev, phost, pesz) : 0;
  if (np < 0) return QED_ERR_ARG;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return QED_ERR_UNSUPPORTED;
  int rc = ensure_host_step(c, per_buf);
  if (rc != QED_OK) return rc;
  // The photons go to the host mirror by a copy kernel writing through
  // host-mapped pointers when every mirror array is mapped (page-locked
  // memory allocated by the CUDA runtime is); otherwise by copies whose
  // ranges the host reads after each chunk.
  PhotonCopy pc{};
  bool mapped = gh != nullptr && np > 0;
  for (int a = 0; a < np && mapped; ++a) {
    void *dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, phost[a], 0) != cudaSuccess) {
      mapped = false;
      cudaGetLastError();  // clear the error of the query
      break;
    }
    pc.src[a] = static_cast<const char *>(pdev[a]);
    pc.dst[a] = static_cast<char *>(dp);
    pc.esz[a] = (int)pesz[a];
    const uintptr_t al = reinterpret_cast<uintptr_t>(pdev[a]) | reinterpret_cast<uintptr_t>(dp);
    pc.wide[a] = al % 16 == 0 ? 16 : al % 4 == 0 ? 4 : 1;
  }
  pc.np = np;
  pc.cap = g->capacity;
  constexpr int R = NBUF + 1;  // device ring of photon counts after each chunk
  int64_t *ring = c->hs_dn + NBUF;
  cudaEvent_t *in_done = c->hs_ev, *comp_done = c->hs_ev + NBUF, *out_done = c->hs_ev + 2 * NBUF;
  int64_t *cnt = c->hs_cnt;  // [0, NBUF): photon count after chunk k (slot k % NBUF); [NBUF]: at start
  cudaError_t e = cudaSuccess;
  int64_t m_done = 0;  // (host-read ranges) photons already on the host mirror
  if (mapped) {
    k_mark_count<<<1, 1, 0, st>>>(ring, g->d_n);
    c->launches += 1;
    e = cudaGetLastError();
  } else {
    e = cudaMemcpyAsync(cnt + NBUF, g->d_n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    m_done = cnt[NBUF];
  }
  if (e != cudaSuccess) return cuda_fail(e, "qed_lepton_step_host");
  const int64_t gcap = g->capacity;
  auto copy_photons = [&](int64_t upto) -> cudaError_t {
    upto = upto < gcap ? upto : gcap;
    if (!gh || upto <= m_done) return cudaSuccess;
    for (int a = 0; a < np; ++a) {
      const size_t o = (size_t)m_done * pesz[a], b = (size_t)(upto - m_done) * pesz[a];
      cudaError_t r = cudaMemcpyAsync(static_cast<char *>(phost[a]) + o,
                                      static_cast<char *>(pdev[a]) + o, b, cudaMemcpyDeviceToHost,
                                      c->hs_out);
      if (r != cudaSuccess) return r;
    }
    m_done = upto;
    return cudaSuccess;
  };
  const int64_t K = (n + chunk - 1) / chunk;
  for (int64_t k = 0; k < K && e == cudaSuccess; ++k) {
    const int b = (int)(k % NBUF);
    const int64_t off = k * chunk, nk = n - off < chunk ? n - off : chunk;
    qed_species sb = staging_species(c, lh, L, nl, b, chunk);
    char *base = static_cast<char *>(c->hs_mem) + (size_t)b * c->hs_per_buf;
    // in: once the buffer's previous chunk has been copied out
    if (k >= NBUF) e = cudaStreamWaitEvent(c->hs_in, out_done[b], 0);
    for (int a = 0; a < nl && e == cudaSuccess; ++a)
      e = cudaMemcpyAsync(base + L[a].off, L[a].host + (size_t)off * L[a].esz, (size_t)nk * L[a].esz,
                          cudaMemcpyHostToDevice, c->hs_in);
    if (e == cudaSuccess) {
      k_set_count<<<1, 1, 0, c->hs_in>>>(c->hs_dn + b, nk);
      c->launches += 1;
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(in_done[b], c->hs_in);
    // step on the caller's stream, then the photon count after it
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, in_done[b], 0);
    if (e == cudaSuccess)
      e = f64 ? launch_lepton<double>(c, &sb, nullptr, g, f, step, MODE_FUSED_, st)
              : launch_lepton<float>(c, &sb, nullptr, g, f, step, MODE_FUSED_, st);
    if (e == cudaSuccess) {
      if (mapped) {
        k_mark_count<<<1, 1, 0, st>>>(ring + (k + 1) % R, g->d_n);
        c->launches += 1;
        e = cudaGetLastError();
      } else {
        e = cudaMemcpyAsync(cnt + b, g->d_n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
      }
    }
    if (e == cudaSuccess) e = cudaEventRecord(comp_done[b], st);
    // out: the updated positions and momenta (and event-generator state), and
    // with mapped mirrors the chunk's photons
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->hs_out, comp_done[b], 0);
    for (int a = 0; a < nl && e == cudaSuccess; ++a)
      if (L[a].back)
        e = cudaMemcpyAsync(L[a].host + (size_t)off * L[a].esz, base + L[a].off, (size_t)nk * L[a].esz,
                            cudaMemcpyDeviceToHost, c->hs_out);
    if (e == cudaSuccess && mapped) {
      // ring slot k % R is rewritten only by chunk k + NBUF, whose input copy
      // waits for this buffer's out_done (recorded after this copy)
      pc.lo = ring + k % R;
      pc.hi = ring + (k + 1) % R;
      k_copy_photons<<<2 * c->num_sms, 256, 0, c->hs_out>>>(pc);
      c->launches += 1;
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(out_done[b], c->hs_out);
    // (host-read ranges) the previous chunk's photons, now that the next
    // chunks are queued
    if (e == cudaSuccess && !mapped && k >= 1) {
      const int pb = (int)((k - 1) % NBUF);
      e = cudaEventSynchronize(comp_done[pb]);
      if (e == cudaSuccess) e = copy_photons(cnt[pb]);
    }
  }
  if (e == cudaSuccess && !mapped && K >= 1) {
    const int lb = (int)((K - 1) % NBUF);
    e = cudaEventSynchronize(comp_done[lb]);
    if (e == cudaSuccess) e = copy_photons(cnt[lb]);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->hs_out);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->hs_in);
  if (e == cudaSuccess && gh && gh->d_n)
    e = cudaMemcpyAsync(cnt + NBUF, g->d_n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "qed_lepton_step_host");
  if (gh && gh->d_n) *gh->d_n = cnt[NBUF] < gcap ? cnt[NBUF] : gcap;
  return QED_OK;
}

}  // namespace qed
