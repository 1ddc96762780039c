// qed_mlp.cu -- training and loading of the surrogate inverse CDF (the
// network is described in qed_mlp.cuh).
//
// Training (qed_mlp_train) runs entirely on the GPU with the project's own
// kernels:
//   k_mlp_grad   each CTA draws mini-batches of (ln chi, kappa) uniformly over
//                the network's domain (Philox), takes the target ln delta from
//                the FP64 inverse table (bicubic, FP64), and runs the forward
//                pass and the hand-written backward pass in FP32 (activations
//                of one mini-batch in shared memory); the CTA's gradient sum
//                goes to its own row of a partial-gradient array;
//   k_mlp_adam   sums the partial rows in a fixed order (deterministic), and
//                applies one bias-corrected Adam step to the FP32 weights;
//   k_mlp_pack   converts W2 and W3 to BF16 tensor-core fragments.
// The loss is the mean squared error of z (ln delta minus its asymptote).
#include <cmath>
#include <cstdio>

#include "qed_internal.h"
#include "qed_mlp.cuh"

namespace qed {

constexpr int GRAD_B = 128;   // samples per mini-batch (one per two threads)
constexpr int GRAD_THREADS = 256;
constexpr int APAD = 65;      // padded row length of the activation arrays

struct GradArgs {
  const float *w;        // FP32 weights
  float *partial;        // [gridDim.x][MLP_NP]
  double *loss_sum;      // [gridDim.x] sum of squared residuals
  // generated batches
  const double *Y64;     // FP64 inverse table (l rows, kappa columns)
  GridR<double> gl, gk;
  uint64_t seed;
  int64_t step;
  int batches_per_cta;
  // explicit batch (gradient checks): x [n][2], t [n]
  const float *x, *t;
  int64_t n;
  float scale;           // dL/dz = scale * (z - t)
};

__device__ __forceinline__ float silu_f(float a) { return a / (1.f + __expf(-a)); }
__device__ __forceinline__ float dsilu_f(float a) {
  float s = 1.f / (1.f + __expf(-a));
  return s * (1.f + a * (1.f - s));
}

__global__ void __launch_bounds__(GRAD_THREADS) k_mlp_grad(GradArgs A) {
  extern __shared__ __align__(16) float sm[];
  float *W = sm;                       // MLP_NP (+3 pad)
  float *G = W + MLP_NP + 3;           // MLP_NP (+3 pad) gradient accumulator
  float *A1 = G + MLP_NP + 3;          // [GRAD_B][APAD]
  float *A2 = A1 + GRAD_B * APAD;
  float *A3 = A2 + GRAD_B * APAD;
  float *X = A3 + GRAD_B * APAD;       // [GRAD_B][2]
  float *T = X + 2 * GRAD_B;           // targets, then dL/dz
  float *Zp = T + GRAD_B;              // half-row output partials
  __shared__ double s_loss[GRAD_THREADS / 32];
  const int tid = threadIdx.x;
  for (int k = tid; k < MLP_NP; k += blockDim.x) {
    W[k] = A.w[k];
    G[k] = 0.f;
  }
  double loss = 0.0;
  const int nb = A.x ? (int)((A.n + (int64_t)GRAD_B * gridDim.x - 1) / ((int64_t)GRAD_B * gridDim.x))
                     : A.batches_per_cta;
  __syncthreads();
  for (int bi = 0; bi < nb; ++bi) {
    const int64_t first = ((int64_t)bi * gridDim.x + blockIdx.x) * GRAD_B;
    // ---- inputs and targets
    if (tid < GRAD_B) {
      float x0 = 0.f, x1 = 0.f, tt = 0.f;
      bool valid = true;
      if (A.x) {
        const int64_t s = first + tid;
        valid = s < A.n;
        if (valid) { x0 = A.x[2 * s]; x1 = A.x[2 * s + 1]; tt = A.t[s]; }
      } else {
        U4 r = philox4x32_10(U4{(uint32_t)(first + tid), (uint32_t)((first + tid) >> 32),
                                (uint32_t)A.step, 0x4D4C5031u},
                             (uint32_t)A.seed, (uint32_t)(A.seed >> 32));
        const double ul = ((double)r.x + 0.5) * 0x1p-32, uk = ((double)r.y + 0.5) * 0x1p-32;
        // the training domain extends past the one the network serves, so
        // that its edges are not the edges of the fit
        const double l = (MLP_L_LO - MLP_TRAIN_DL) + (MLP_L_HI - MLP_L_LO + 2 * MLP_TRAIN_DL) * ul;
        const double k = (MLP_K_LO - MLP_TRAIN_DK) + (MLP_K_HI - MLP_K_LO + 2 * MLP_TRAIN_DK) * uk;
        const double Y = interp2(A.Y64, A.gl, l, A.gk, k);
        const double sp = k > 30.0 ? k : log1p(exp(k));
        x0 = (float)((l - MLP_LC) / MLP_LS);
        x1 = (float)((k - MLP_KC) / MLP_KS);
        tt = (float)(Y - (3.0 * k - 2.0 * sp));
      }
      X[2 * tid] = x0;
      X[2 * tid + 1] = x1;
      T[tid] = valid ? tt : NAN;  // NaN marks a padding row (no gradient)
    }
    __syncthreads();
    // ---- forward: A1 = X W1 + b1 ; thread -> (row = tid % 128, column half = tid / 128)
    const int row = tid % GRAD_B, c0 = (tid / GRAD_B) * 32;
    for (int c = c0; c < c0 + 32; ++c)
      A1[row * APAD + c] = fmaf(X[2 * row], W[MLP_OFF_W1 + c],
                                fmaf(X[2 * row + 1], W[MLP_OFF_W1 + 64 + c], W[MLP_OFF_B1 + c]));
    __syncthreads();
    {
      float acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = W[MLP_OFF_B2 + c0 + j];
      for (int k = 0; k < 64; ++k) {
        const float h = silu_f(A1[row * APAD + k]);
        const float *wr = W + MLP_OFF_W2 + k * 64 + c0;
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = fmaf(h, wr[j], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) A2[row * APAD + c0 + j] = acc[j];
    }
    __syncthreads();
    {
      float acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = W[MLP_OFF_B3 + c0 + j];
      for (int k = 0; k < 64; ++k) {
        const float h = silu_f(A2[row * APAD + k]);
        const float *wr = W + MLP_OFF_W3 + k * 64 + c0;
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = fmaf(h, wr[j], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) A3[row * APAD + c0 + j] = acc[j];
    }
    __syncthreads();
    // ---- output and dL/dz (two threads per row: column halves combined in shared memory)
    {
      float part = 0.f;
      for (int c = c0; c < c0 + 32; ++c) part = fmaf(silu_f(A3[row * APAD + c]), W[MLP_OFF_W4 + c], part);
      if (tid >= GRAD_B) Zp[row] = part;
      __syncthreads();
      if (tid < GRAD_B) {
        const float z = part + Zp[row] + W[MLP_OFF_B4];
        const float tt = T[row];
        float dz = 0.f;
        if (!isnan(tt)) {
          const float r = z - tt;
          loss += (double)r * r;
          dz = A.scale * r;
        }
        T[row] = dz;
      }
      __syncthreads();
    }
    // ---- backward
    // W4, b4 (one thread per column, rows summed in order)
    if (tid < 64) {
      float gw = 0.f;
      for (int r = 0; r < GRAD_B; ++r) gw = fmaf(silu_f(A3[r * APAD + tid]), T[r], gw);
      G[MLP_OFF_W4 + tid] += gw;
    } else if (tid == 64) {
      float gb = 0.f;
      for (int r = 0; r < GRAD_B; ++r) gb += T[r];
      G[MLP_OFF_B4] += gb;
    }
    __syncthreads();
    // dA3 = dz * W4 * silu'(A3), in place
    for (int c = c0; c < c0 + 32; ++c)
      A3[row * APAD + c] = T[row] * W[MLP_OFF_W4 + c] * dsilu_f(A3[row * APAD + c]);
    __syncthreads();
    // gW3[j][k] = sum_r h2[r][j] dA3[r][k]; gb3[k] = sum_r dA3[r][k]
    {
      const int j = tid / 4, kb = (tid % 4) * 16;
      float acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = 0.f;
      for (int r = 0; r < GRAD_B; ++r) {
        const float h = silu_f(A2[r * APAD + j]);
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = fmaf(h, A3[r * APAD + kb + q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) G[MLP_OFF_W3 + j * 64 + kb + q] += acc[q];
    }
    if (tid < 64) {
      float gb = 0.f;
      for (int r = 0; r < GRAD_B; ++r) gb += A3[r * APAD + tid];
      G[MLP_OFF_B3 + tid] += gb;
    }
    __syncthreads();
    // dH2 = dA3 W3^T ; dA2 = dH2 * silu'(A2) (in place)
    {
      float acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0.f;
      for (int k = 0; k < 64; ++k) {
        const float d = A3[row * APAD + k];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = fmaf(d, W[MLP_OFF_W3 + (c0 + j) * 64 + k], acc[j]);
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = c0 + j;
        A2[row * APAD + c] = acc[j] * dsilu_f(A2[row * APAD + c]);
      }
    }
    __syncthreads();
    // gW2, gb2 from h1 = silu(A1) and dA2
    {
      const int j = tid / 4, kb = (tid % 4) * 16;
      float acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = 0.f;
      for (int r = 0; r < GRAD_B; ++r) {
        const float h = silu_f(A1[r * APAD + j]);
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = fmaf(h, A2[r * APAD + kb + q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) G[MLP_OFF_W2 + j * 64 + kb + q] += acc[q];
    }
    if (tid < 64) {
      float gb = 0.f;
      for (int r = 0; r < GRAD_B; ++r) gb += A2[r * APAD + tid];
      G[MLP_OFF_B2 + tid] += gb;
    }
    __syncthreads();
    // dH1 = dA2 W2^T ; dA1 = dH1 * silu'(A1) (in place)
    {
      float acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0.f;
      for (int k = 0; k < 64; ++k) {
        const float d = A2[row * APAD + k];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = fmaf(d, W[MLP_OFF_W2 + (c0 + j) * 64 + k], acc[j]);
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = c0 + j;
        A1[row * APAD + c] = acc[j] * dsilu_f(A1[row * APAD + c]);
      }
    }
    __syncthreads();
    // gW1[i][k] = sum_r x[r][i] dA1[r][k] ; gb1[k] = sum_r dA1[r][k]
    if (tid < 192) {
      const int k = tid % 64, which = tid / 64;  // 0: W1 row 0, 1: W1 row 1, 2: b1
      float acc = 0.f;
      for (int r = 0; r < GRAD_B; ++r) {
        const float d = A1[r * APAD + k];
        const float f = which == 2 ? 1.f : X[2 * r + which];
        acc = fmaf(f, d, acc);
      }
      if (which == 2) G[MLP_OFF_B1 + k] += acc;
      else G[MLP_OFF_W1 + which * 64 + k] += acc;
    }
    __syncthreads();
  }
  for (int k = tid; k < MLP_NP; k += blockDim.x) A.partial[(size_t)blockIdx.x * MLP_NP + k] = G[k];
  // loss of this CTA
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if ((tid & 31) == 0) s_loss[tid >> 5] = loss;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < GRAD_THREADS / 32; ++w) s += s_loss[w];
    A.loss_sum[blockIdx.x] = s;
  }
}

struct AdamArgs {
  float *w, *m, *v;
  const float *partial;
  int nparts;
  float lr, b1, b2, eps, bc1, bc2;
  float *grad_out;  // optional: the summed gradient (gradient checks)
  int apply;
};

__global__ void k_mlp_adam(AdamArgs A) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= MLP_NP) return;
  float g = 0.f;
  for (int p = 0; p < A.nparts; ++p) g += A.partial[(size_t)p * MLP_NP + k];  // fixed order
  if (A.grad_out) A.grad_out[k] = g;
  if (!A.apply) return;
  const float m = A.b1 * A.m[k] + (1.f - A.b1) * g;
  const float v = A.b2 * A.v[k] + (1.f - A.b2) * g * g;
  A.m[k] = m;
  A.v[k] = v;
  A.w[k] -= A.lr * (m / A.bc1) / (sqrtf(v / A.bc2) + A.eps);
}

// BF16 B fragments of W2 and W3 for mma.sync m16n8k16 (B = W, K x N): the
// high parts, then the remainders W - hi (see qed_mlp.cuh).
__device__ __forceinline__ void pack_split(float a, float b, uint32_t &hi, uint32_t &lo) {
  split_bf16(a, b, hi, lo);
}

__global__ void k_mlp_pack(const float *w, uint32_t *frag) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // over [layer][kt][nt][lane]
  if (idx >= 2 * 4 * 8 * 32) return;
  const int lane = idx & 31, nt = (idx >> 5) & 7, kt = (idx >> 8) & 3, layer = idx >> 10;
  const float *W = w + (layer ? MLP_OFF_W3 : MLP_OFF_W2);
  const int g = lane >> 2, t = lane & 3, n = nt * 8 + g;
  const int k0 = kt * 16 + 2 * t;
  uint32_t *F = frag + layer * MLP_FRAG_LAYER;
  uint32_t *Fl = F + MLP_FRAG_LAYER / 2;
  const int o = 2 * (idx & 1023);
  pack_split(W[k0 * 64 + n], W[(k0 + 1) * 64 + n], F[o], Fl[o]);
  pack_split(W[(k0 + 8) * 64 + n], W[(k0 + 9) * 64 + n], F[o + 1], Fl[o + 1]);
}

static size_t grad_smem() {
  return sizeof(float) * (2 * (MLP_NP + 3) + 3 * GRAD_B * APAD + 4 * GRAD_B);
}

int mlp_alloc(qed_ctx *c) {
  c->mlp_parts = c->num_sms;
  size_t bytes = sizeof(float) * MLP_NP * 4 + sizeof(uint32_t) * MLP_FRAG_WORDS +
                 sizeof(float) * MLP_SMEM_FLOATS + sizeof(float) * (size_t)MLP_NP * c->mlp_parts +
                 sizeof(double) * c->mlp_parts;
  if (cudaMalloc(&c->mlp_mem, bytes) != cudaSuccess) return QED_ERR_NOMEM;
  float *f = static_cast<float *>(c->mlp_mem);
  c->mlp_w = f;
  c->mlp_m = f + MLP_NP;
  c->mlp_v = f + 2 * MLP_NP;
  c->mlp_g = f + 3 * MLP_NP;
  c->mlp_frag = reinterpret_cast<uint32_t *>(f + 4 * MLP_NP);
  c->mlp_fw = reinterpret_cast<float *>(c->mlp_frag + MLP_FRAG_WORDS);
  c->mlp_partial = c->mlp_fw + MLP_SMEM_FLOATS;
  c->mlp_loss = reinterpret_cast<double *>(c->mlp_partial + (size_t)MLP_NP * c->mlp_parts);
  if (cudaMemset(c->mlp_mem, 0, bytes) != cudaSuccess) return QED_ERR_CUDA;
  if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)grad_smem()) != cudaSuccess)
    return QED_ERR_CUDA;
  c->mlp_ready = 0;
  c->mlp_step = 0;
  // records of deferred learned-sampler emissions (single-pass lepton step of
  // an FP32 context with the learned sampler): 16 bytes (48 with grid
  // fields) per emission, at most one per lepton at step start.  Two species
  // of at most max_particles each fill 2 max_particles records of 16 bytes;
  // with grid fields two thirds of that, while a one-sub-step lepton emits
  // with probability <= 0.2 (a record past the end is counted as dropped).
  c->net_cap = 0;
  if (c->cfg.sampler != QED_SAMPLER_MLP || c->cfg.append_order != QED_APPEND_ANY ||
      c->cfg.precision != QED_FP32)
    return QED_OK;
  c->net_cap = 2 * (c->cfg.max_particles > 4096 ? c->cfg.max_particles : 4096);
  if (cudaMalloc(&c->net_rec, sizeof(float4) * (size_t)c->net_cap) != cudaSuccess ||
      cudaMalloc(&c->net_n, 2 * sizeof(unsigned long long)) != cudaSuccess)
    return QED_ERR_NOMEM;
  if (cudaMemset(c->net_n, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) return QED_ERR_CUDA;
  return QED_OK;
}

// The FP32 small layers in the layout inference reads (as staged by mlp_stage).
__global__ void k_mlp_pack_fw(const float *w, float *fw) {
  for (int k = threadIdx.x; k < MLP_SMEM_FLOATS; k += blockDim.x) {
    float v = 0.f;
    if (k < 128) v = w[MLP_OFF_W1 + k];
    else if (k < 192) v = w[MLP_OFF_B1 + k - 128];
    else if (k < 256) v = w[MLP_OFF_B2 + k - 192];
    else if (k < 320) v = w[MLP_OFF_B3 + k - 256];
    else if (k < 384) v = w[MLP_OFF_W4 + k - 320];
    else if (k == 384) v = w[MLP_OFF_B4];
    fw[k] = v;
  }
}

static cudaError_t pack(qed_ctx *c, cudaStream_t st) {
  k_mlp_pack<<<(2 * 4 * 8 * 32 + 255) / 256, 256, 0, st>>>(c->mlp_w, c->mlp_frag);
  k_mlp_pack_fw<<<1, 128, 0, st>>>(c->mlp_w, c->mlp_fw);
  c->launches += 2;
  return cudaGetLastError();
}

static GradArgs grad_args(qed_ctx *c) {
  GradArgs g{};
  g.w = c->mlp_w;
  g.partial = c->mlp_partial;
  g.loss_sum = c->mlp_loss;
  g.Y64 = c->Y64;
  g.gl = to_r<double>(c->gl);
  g.gk = to_r<double>(c->gk);
  return g;
}

}  // namespace qed

using namespace qed;

static int fail(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return QED_OK;
  fprintf(stderr, "libqed: %s: %s\n", what, cudaGetErrorString(e));
  return QED_ERR_CUDA;
}

extern "C" int qed_mlp_load(qed_ctx *c, const float *host_w, size_t n) {
  if (!c || !host_w || n != (size_t)MLP_NP) return QED_ERR_ARG;
  cudaError_t e = cudaMemcpy(c->mlp_w, host_w, sizeof(float) * MLP_NP, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->mlp_m, 0, sizeof(float) * 2 * MLP_NP);
  if (e == cudaSuccess) e = pack(c, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(e, "qed_mlp_load");
  c->mlp_ready = 1;
  c->mlp_step = 0;
  return QED_OK;
}

extern "C" int qed_mlp_get(qed_ctx *c, float *host_w, size_t n) {
  if (!c || !host_w || n != (size_t)MLP_NP) return QED_ERR_ARG;
  return fail(cudaMemcpy(host_w, c->mlp_w, sizeof(float) * MLP_NP, cudaMemcpyDeviceToHost),
              "qed_mlp_get");
}

extern "C" int qed_mlp_grad(qed_ctx *c, const float *x, const float *t, int64_t n, float *grad,
                            double *loss, qed_stream_t stream) {
  if (!c || !x || !t || !grad || n <= 0) return QED_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  GradArgs g = grad_args(c);
  g.x = x;
  g.t = t;
  g.n = n;
  g.scale = 2.f / (float)n;
  k_mlp_grad<<<c->mlp_parts, GRAD_THREADS, grad_smem(), st>>>(g);
  AdamArgs a{};
  a.w = c->mlp_w;
  a.partial = c->mlp_partial;
  a.nparts = c->mlp_parts;
  a.grad_out = grad;
  a.apply = 0;
  k_mlp_adam<<<(MLP_NP + 255) / 256, 256, 0, st>>>(a);
  c->launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && loss) {
    double tmp[1024];
    int np = c->mlp_parts < 1024 ? c->mlp_parts : 1024;
    e = cudaMemcpyAsync(tmp, c->mlp_loss, sizeof(double) * np, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    double s = 0.0;
    for (int p = 0; p < np; ++p) s += tmp[p];
    *loss = s / (double)n;
  }
  return fail(e, "qed_mlp_grad");
}

extern "C" int qed_mlp_train(qed_ctx *c, int64_t n_samples, float lr, uint64_t seed,
                             double *final_loss, qed_stream_t stream) {
  if (!c || n_samples <= 0 || !(lr > 0.f)) return QED_ERR_ARG;
  if (!c->mlp_ready) return QED_ERR_ARG;  // initial weights must be loaded first
  cudaStream_t st = (cudaStream_t)stream;
  const int bpc = 2;  // mini-batches per CTA per optimizer step
  const int64_t per_step = (int64_t)GRAD_B * bpc * c->mlp_parts;
  const int64_t steps = (n_samples + per_step - 1) / per_step;
  GradArgs g = grad_args(c);
  g.seed = seed;
  g.batches_per_cta = bpc;
  g.scale = 2.f / (float)per_step;
  AdamArgs a{};
  a.w = c->mlp_w;
  a.m = c->mlp_m;
  a.v = c->mlp_v;
  a.partial = c->mlp_partial;
  a.nparts = c->mlp_parts;
  a.b1 = 0.9f;
  a.b2 = 0.999f;
  a.eps = 1e-8f;
  a.apply = 1;
  const float lr_min = lr * 0.01f;
  double loss_tail = 0.0;
  int64_t tail_n = 0;
  for (int64_t s = 0; s < steps; ++s) {
    g.step = c->mlp_step + s;
    k_mlp_grad<<<c->mlp_parts, GRAD_THREADS, grad_smem(), st>>>(g);
    const int64_t k = c->mlp_step + s + 1;  // Adam step count (from 1)
    a.lr = lr_min + 0.5f * (lr - lr_min) * (1.f + cosf(3.14159265f * (float)s / (float)steps));
    a.bc1 = 1.f - powf(a.b1, (float)k);
    a.bc2 = 1.f - powf(a.b2, (float)k);
    k_mlp_adam<<<(MLP_NP + 255) / 256, 256, 0, st>>>(a);
    c->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(e, "qed_mlp_train");
    if (s >= steps - 8) {  // mean loss of the last steps (synchronises only there)
      double tmp[1024];
      int np = c->mlp_parts < 1024 ? c->mlp_parts : 1024;
      e = cudaMemcpyAsync(tmp, c->mlp_loss, sizeof(double) * np, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return fail(e, "qed_mlp_train");
      double sum = 0.0;
      for (int p = 0; p < np; ++p) sum += tmp[p];
      loss_tail += sum / (double)per_step;
      tail_n += 1;
    }
  }
  c->mlp_step += steps;
  cudaError_t e = pack(c, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (final_loss) *final_loss = tail_n ? loss_tail / tail_n : 0.0;
  return fail(e, "qed_mlp_train");
}
