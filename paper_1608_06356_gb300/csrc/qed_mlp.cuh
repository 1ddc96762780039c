// qed_mlp.cuh -- the surrogate inverse CDF: a 2 -> 64 -> 64 -> 64 -> 1 SiLU
// network that maps (ln chi, kappa) to ln delta for photon emission, where
// kappa = ln(-ln(1-u)) and delta = 2 xi / (3 chi (1 - xi)) (the coordinates of
// the tabulated inverse of Eq. (7)).
//
//   x0 = (ln chi - MLP_LC) / MLP_LS,  x1 = (kappa - MLP_KC) / MLP_KS
//   z  = network(x0, x1),             ln delta = z + 3 kappa - 2 softplus(kappa)
//
// (3 kappa - 2 softplus(kappa) is the two-sided asymptote of ln delta, so z
// stays O(1).)  Domain: chi in [1e-3, 1e2], kappa in [-10, 3.5]; outside it
// the table sampler is used.  Parameters (FP32, 8577 values) are laid out as
// W1[2][64], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4.
// Inference runs layers 2 and 3 on the tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation).  Each operand is split into a BF16 high part
// and a BF16 remainder, and a tile product is accumulated as
// hi*hi + lo*hi + hi*lo (three MMAs), which carries ~16 significant bits --
// single BF16 operands (8 bits) would move sampled photon energies by ~1%.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace qed {

constexpr int MLP_H = 64;
constexpr int MLP_NP = 8577;
constexpr int MLP_OFF_W1 = 0, MLP_OFF_B1 = 128, MLP_OFF_W2 = 192, MLP_OFF_B2 = 4288,
              MLP_OFF_W3 = 4352, MLP_OFF_B3 = 8448, MLP_OFF_W4 = 8512, MLP_OFF_B4 = 8576;
// input normalisation: ln chi over [ln 1e-3, ln 1e2], kappa over [-10, 3.5]
constexpr float MLP_LC = -1.1512925465f;  // (ln 1e-3 + ln 1e2) / 2
constexpr float MLP_LS = 5.7564627325f;   // (ln 1e2 - ln 1e-3) / 2
constexpr float MLP_KC = -3.25f, MLP_KS = 6.75f;
constexpr float MLP_L_LO = -6.9077552790f, MLP_L_HI = 4.6051701860f;
constexpr float MLP_K_LO = -10.0f, MLP_K_HI = 3.5f;
// margins of the training domain beyond the served one, in ln chi and kappa
constexpr double MLP_TRAIN_DL = 0.3, MLP_TRAIN_DK = 0.25;
// BF16 fragments of W2 and W3: [layer 2][hi/lo 2][kt 4][nt 8][lane 32][2] uint32
constexpr int MLP_FRAG_LAYER = 2 * 4 * 8 * 32 * 2;
constexpr int MLP_FRAG_WORDS = 2 * MLP_FRAG_LAYER;
// shared-memory image used by inference: fragments + FP32 W1, b1, b2, b3, W4, b4
constexpr int MLP_SMEM_FLOATS = 128 + 64 + 64 + 64 + 64 + 1 + 3;  // padded to 16 B
constexpr size_t MLP_SMEM_BYTES = MLP_FRAG_WORDS * 4 + MLP_SMEM_FLOATS * 4;

__device__ __forceinline__ float mlp_baseline(float k) {
  // 3k - 2 softplus(k)
  float sp = k > 15.f ? k : log1pf(__expf(k));
  return 3.f * k - 2.f * sp;
}

// SiLU with the fast exponential and the fast division (two SFU operations
// and a multiply; a few ulp, far below the split-BF16 products' 1e-5)
__device__ __forceinline__ float silu_fast(float x) { return __fdividef(x, 1.f + __expf(-x)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

// (x0, x1) -> BF16 pair of the high parts and BF16 pair of the remainders.
__device__ __forceinline__ void split_bf16(float x0, float x1, uint32_t &hi, uint32_t &lo) {
  __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  float2 hf = __bfloat1622float2(h);
  hi = *reinterpret_cast<uint32_t *>(&h);
  lo = pack_bf16(x0 - hf.x, x1 - hf.y);
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], uint32_t b0,
                                               uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Warp-collective inference: every lane passes its sample's (x0, x1) and gets
// z back.  All 32 lanes must call it.  frag: BF16 fragments (shared memory);
// fw: FP32 W1 (128), b1, b2, b3, W4 (64 each), b4 (shared memory).
__device__ __forceinline__ float mlp_infer_warp(const uint32_t *frag, const float *fw, float x0,
                                                float x1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const float *W1 = fw, *b1 = fw + 128, *b2 = fw + 192, *b3 = fw + 256, *W4 = fw + 320;
  const float b4 = fw[384];
  float out_lo[2], out_hi[2];
  // the two 16-sample tiles run as a loop (not unrolled): the body is large
  // and is inlined into the step kernels, whose instruction cache it shares
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    // inputs of rows g and g+8 of this 16-sample tile
    const float xa0 = __shfl_sync(0xffffffffu, x0, mt * 16 + g);
    const float xa1 = __shfl_sync(0xffffffffu, x1, mt * 16 + g);
    const float xb0 = __shfl_sync(0xffffffffu, x0, mt * 16 + g + 8);
    const float xb1 = __shfl_sync(0xffffffffu, x1, mt * 16 + g + 8);
    // layer 1 (K = 2, CUDA cores), written straight into layer-2 A fragments
    uint32_t A[4][4], Al[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int c = kt * 16 + half * 8 + 2 * t;
        float r0c0 = silu_fast(fmaf(xa0, W1[c], fmaf(xa1, W1[64 + c], b1[c])));
        float r0c1 = silu_fast(fmaf(xa0, W1[c + 1], fmaf(xa1, W1[64 + c + 1], b1[c + 1])));
        float r1c0 = silu_fast(fmaf(xb0, W1[c], fmaf(xb1, W1[64 + c], b1[c])));
        float r1c1 = silu_fast(fmaf(xb0, W1[c + 1], fmaf(xb1, W1[64 + c + 1], b1[c + 1])));
        split_bf16(r0c0, r0c1, A[kt][half * 2 + 0], Al[kt][half * 2 + 0]);
        split_bf16(r1c0, r1c1, A[kt][half * 2 + 1], Al[kt][half * 2 + 1]);
      }
    }
    // layers 2 and 3 on the tensor cores
    const float *bias[2] = {b2, b3};
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {
      const uint32_t *F = frag + layer * MLP_FRAG_LAYER;       // high parts
      const uint32_t *Fl = F + MLP_FRAG_LAYER / 2;              // remainders
      uint32_t An[4][4], Anl[4][4];
      float acc4_lo = 0.f, acc4_hi = 0.f;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int c = nt * 8 + 2 * t;
        float acc[4] = {bias[layer][c], bias[layer][c + 1], bias[layer][c], bias[layer][c + 1]};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
          const int o = ((kt * 8 + nt) * 32 + lane) * 2;
          const uint2 b = *reinterpret_cast<const uint2 *>(F + o);
          const uint2 bl = *reinterpret_cast<const uint2 *>(Fl + o);
          mma_bf16_16816(acc, Al[kt], b.x, b.y);
          mma_bf16_16816(acc, A[kt], bl.x, bl.y);
          mma_bf16_16816(acc, A[kt], b.x, b.y);
        }
        const float h0 = silu_fast(acc[0]), h1 = silu_fast(acc[1]);
        const float h2 = silu_fast(acc[2]), h3 = silu_fast(acc[3]);
        if (layer == 0) {
          // C layout of n-tile nt = A layout of k-tile nt/2 (left or right half)
          split_bf16(h0, h1, An[nt >> 1][(nt & 1) * 2 + 0], Anl[nt >> 1][(nt & 1) * 2 + 0]);
          split_bf16(h2, h3, An[nt >> 1][(nt & 1) * 2 + 1], Anl[nt >> 1][(nt & 1) * 2 + 1]);
        } else {
          // layer 4 (64 -> 1) partial dot products for rows g and g+8
          acc4_lo = fmaf(h0, W4[c], fmaf(h1, W4[c + 1], acc4_lo));
          acc4_hi = fmaf(h2, W4[c], fmaf(h3, W4[c + 1], acc4_hi));
        }
      }
      if (layer == 0) {
#pragma unroll
        for (int kt = 0; kt < 4; ++kt)
#pragma unroll
          for (int r = 0; r < 4; ++r) { A[kt][r] = An[kt][r]; Al[kt][r] = Anl[kt][r]; }
      } else {
        acc4_lo += __shfl_xor_sync(0xffffffffu, acc4_lo, 1);
        acc4_lo += __shfl_xor_sync(0xffffffffu, acc4_lo, 2);
        acc4_hi += __shfl_xor_sync(0xffffffffu, acc4_hi, 1);
        acc4_hi += __shfl_xor_sync(0xffffffffu, acc4_hi, 2);
        out_lo[mt] = acc4_lo + b4;
        out_hi[mt] = acc4_hi + b4;
      }
    }
  }
  // sample s = mt*16 + r lives in lanes 4*(r%8).. as out_lo (r < 8) or out_hi (r >= 8)
  const int mt = lane >> 4, r = lane & 15;
  const int src = 4 * (r & 7);
  float lo0 = __shfl_sync(0xffffffffu, out_lo[0], src), hi0 = __shfl_sync(0xffffffffu, out_hi[0], src);
  float lo1 = __shfl_sync(0xffffffffu, out_lo[1], src), hi1 = __shfl_sync(0xffffffffu, out_hi[1], src);
  float lo = mt ? lo1 : lo0, hi = mt ? hi1 : hi0;
  return r < 8 ? lo : hi;
}

// Stage the inference image (fragments + FP32 small layers) into shared memory.
__device__ __forceinline__ void mlp_stage(uint32_t *s_frag, float *s_fw, const uint32_t *frag,
                                          const float *w) {
  for (int k = threadIdx.x; k < MLP_FRAG_WORDS; k += blockDim.x) s_frag[k] = frag[k];
  for (int k = threadIdx.x; k < 128; k += blockDim.x) s_fw[k] = w[MLP_OFF_W1 + k];
  for (int k = threadIdx.x; k < 64; k += blockDim.x) {
    s_fw[128 + k] = w[MLP_OFF_B1 + k];
    s_fw[192 + k] = w[MLP_OFF_B2 + k];
    s_fw[256 + k] = w[MLP_OFF_B3 + k];
    s_fw[320 + k] = w[MLP_OFF_W4 + k];
  }
  if (threadIdx.x == 0) s_fw[384] = w[MLP_OFF_B4];
}

}  // namespace qed
