// mlp_kernels.cuh -- learned lane-change surrogate: 16 -> 64 -> 64 -> 3 MLP on the tensor
// cores (BF16 operands, FP32 accumulation).  The paper's lane-change model is rule-based
// (MOBIL, Sec. III-A); this network is the library's learned replacement of the MOBIL
// incentive decision, trained on decisions logged from the rule-based step.
//
// Parameter vector (FP32 master copy, 5443 floats): W1[64][16], b1[64], W2[64][64], b2[64],
// W3[3][64], b3[3] (row-major, out x in).  Device model for inference / training operands:
// BF16 W1, W2, W3 padded to 16 rows, FP32 biases (see MlpDev).
//
// Tensor-core primitive: mma.sync m16n8k16 (row.col, bf16 x bf16 -> f32), operand
// fragments assembled from shared memory by each lane (PTX ISA fragment layout: lane l
// holds rows g = l/4 and g + 8, columns / k indices 2*(l%4) + {0,1} and + 8).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "umma.cuh"

namespace moss {

constexpr int MLP_IN = 16, MLP_H = 64, MLP_OUT = 3, MLP_OUTP = 16;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H,
              OFF_B2 = OFF_W2 + MLP_H * MLP_H, OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_OUT * MLP_H;

// BF16 operands + FP32 biases, as laid out in global and shared memory
struct MlpDev {
  __nv_bfloat16 w1[MLP_H * MLP_IN];     // [64][16]
  __nv_bfloat16 w2[MLP_H * MLP_H];      // [64][64]
  __nv_bfloat16 w3[MLP_OUTP * MLP_H];   // [16][64], rows 3..15 zero
  float b1[MLP_H], b2[MLP_H], b3[MLP_OUTP];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  __nv_bfloat162 h;
  h.x = lo;
  h.y = hi;
  return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment of a 16x16 tile whose element (m, k) is A(m, k)
template <class FA>
__device__ __forceinline__ void load_a(uint32_t a[4], FA A) {
  const int l = threadIdx.x & 31, g = l >> 2, t = (l & 3) * 2;
  a[0] = pack2(A(g, t), A(g, t + 1));
  a[1] = pack2(A(g + 8, t), A(g + 8, t + 1));
  a[2] = pack2(A(g, t + 8), A(g, t + 9));
  a[3] = pack2(A(g + 8, t + 8), A(g + 8, t + 9));
}

// B fragment of a 16x8 tile whose element (k, n) is B(k, n)
template <class FB>
__device__ __forceinline__ void load_b(uint32_t b[2], FB B) {
  const int l = threadIdx.x & 31, g = l >> 2, t = (l & 3) * 2;
  b[0] = pack2(B(t, g), B(t + 1, g));
  b[1] = pack2(B(t + 8, g), B(t + 9, g));
}

// The same fragments from row-major bf16 storage with k contiguous: A(m, k) = A[m * lda + k],
// B(k, n) = W[(n0 + n) * ldw + k0 + k] (a weight matrix stored [out][in]).  Each register
// holds two k-adjacent elements, so it is one 32-bit shared-memory load (lda, ldw, k0 even).
__device__ __forceinline__ void load_a_rm(uint32_t a[4], const __nv_bfloat16 *A, int lda) {
  const int l = threadIdx.x & 31, g = l >> 2, t = (l & 3) * 2;
  a[0] = *reinterpret_cast<const uint32_t *>(A + g * lda + t);
  a[1] = *reinterpret_cast<const uint32_t *>(A + (g + 8) * lda + t);
  a[2] = *reinterpret_cast<const uint32_t *>(A + g * lda + t + 8);
  a[3] = *reinterpret_cast<const uint32_t *>(A + (g + 8) * lda + t + 8);
}
__device__ __forceinline__ void load_b_nk(uint32_t b[2], const __nv_bfloat16 *W, int ldw, int n0, int k0) {
  const int l = threadIdx.x & 31, g = l >> 2, t = (l & 3) * 2;
  const __nv_bfloat16 *r = W + (n0 + g) * ldw + k0 + t;
  b[0] = *reinterpret_cast<const uint32_t *>(r);
  b[1] = *reinterpret_cast<const uint32_t *>(r + 8);
}

// Store a 16x8 accumulator tile through f(m, n, value)
template <class FC>
__device__ __forceinline__ void store_c(const float c[4], FC f) {
  const int l = threadIdx.x & 31, g = l >> 2, t = (l & 3) * 2;
  f(g, t, c[0]);
  f(g, t + 1, c[1]);
  f(g + 8, t, c[2]);
  f(g + 8, t + 1, c[3]);
}

// Forward of 16 rows (one m-tile) by one warp.  X: [16][16] bf16 (row stride 16), H1:
// [16][64] bf16 scratch (row stride 64), out: logits [16][MLP_OUT] fp32 written through f.
// Optionally keeps H2 ([16][64] bf16) for the backward pass.
template <class FO>
__device__ __forceinline__ void mlp_forward_tile(const MlpDev &w, const __nv_bfloat16 *X, __nv_bfloat16 *H1,
                                                 __nv_bfloat16 *H2, FO out) {
  uint32_t a[4], b[2];
  // layer 1: [16 x 16] x W1^T -> [16 x 64]
  load_a_rm(a, X, MLP_IN);
#pragma unroll
  for (int nt = 0; nt < MLP_H / 8; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    load_b_nk(b, w.w1, MLP_IN, nt * 8, 0);
    mma16816(c, a, b);
    store_c(c, [&](int m, int n, float v) {
      H1[m * MLP_H + nt * 8 + n] = __float2bfloat16_rn(fmaxf(v + w.b1[nt * 8 + n], 0.f));
    });
  }
  __syncwarp();
  // layer 2 -> register chunks of 16 columns, each fed straight into layer 3 as an A fragment
  float z[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
  for (int ch = 0; ch < MLP_H / 16; ++ch) {
    float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int ks = 0; ks < MLP_H / 16; ++ks) {
      load_a_rm(a, H1 + ks * 16, MLP_H);
      load_b_nk(b, w.w2, MLP_H, ch * 16, ks * 16);
      mma16816(c0, a, b);
      load_b_nk(b, w.w2, MLP_H, ch * 16 + 8, ks * 16);
      mma16816(c1, a, b);
    }
    // bias + ReLU; accumulator layout of two 8-column tiles == A fragment of one 16-wide k step
    const int l = threadIdx.x & 31, t = (l & 3) * 2;
    const float b00 = w.b2[ch * 16 + t], b01 = w.b2[ch * 16 + t + 1];
    const float b10 = w.b2[ch * 16 + 8 + t], b11 = w.b2[ch * 16 + 9 + t];
    float h[8] = {fmaxf(c0[0] + b00, 0.f), fmaxf(c0[1] + b01, 0.f), fmaxf(c0[2] + b00, 0.f),
                  fmaxf(c0[3] + b01, 0.f), fmaxf(c1[0] + b10, 0.f), fmaxf(c1[1] + b11, 0.f),
                  fmaxf(c1[2] + b10, 0.f), fmaxf(c1[3] + b11, 0.f)};
    uint32_t ah[4] = {pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]),
                      pack_bf16(h[6], h[7])};
    if (H2) {
      const int g = l >> 2;
      H2[g * MLP_H + ch * 16 + t] = __float2bfloat16_rn(h[0]);
      H2[g * MLP_H + ch * 16 + t + 1] = __float2bfloat16_rn(h[1]);
      H2[(g + 8) * MLP_H + ch * 16 + t] = __float2bfloat16_rn(h[2]);
      H2[(g + 8) * MLP_H + ch * 16 + t + 1] = __float2bfloat16_rn(h[3]);
      H2[g * MLP_H + ch * 16 + 8 + t] = __float2bfloat16_rn(h[4]);
      H2[g * MLP_H + ch * 16 + 9 + t] = __float2bfloat16_rn(h[5]);
      H2[(g + 8) * MLP_H + ch * 16 + 8 + t] = __float2bfloat16_rn(h[6]);
      H2[(g + 8) * MLP_H + ch * 16 + 9 + t] = __float2bfloat16_rn(h[7]);
    }
    // layer 3: this 16-wide slice of h2 times W3 (padded to 16 outputs = two n-tiles)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      load_b_nk(b, w.w3, MLP_H, nt * 8, ch * 16);
      mma16816(z[nt], ah, b);
    }
  }
  store_c(z[0], [&](int m, int n, float v) {
    if (n < MLP_OUT) out(m, n, v + w.b3[n]);
  });
}

// ------------------------------------------------------------------------------------
// training
// ------------------------------------------------------------------------------------

constexpr int TR_ROWS = 64;             // samples per block
constexpr int TR_WARPS = TR_ROWS / 16;  // one m-tile per warp

struct TrainArgs {
  const __nv_bfloat16 *X;   // [n][16] features
  const int *y;             // [n] labels 0..2
  const int *idx;           // [batch] sample indices of this minibatch
  int batch;
  const MlpDev *model;      // BF16 operands of the current parameters
  float cw[3];              // class weights
  float *grad;              // [MLP_NPARAM] accumulated, unnormalised
  float *stats;             // [0] sum of weights, [1] weighted loss sum
  unsigned *err;            // k_mlp_train_tc: set when a wait for the tensor core ran out
  const float *theta;       // k_mlp_train_tc: FP32 parameters, from which it packs its operands
  int withhold;             // test of the timeout path: no MMA is issued or committed, so the
                            // first wait runs out (after a short limit) and sets err
};

// One Adam step (Kingma & Ba 2015) of parameter k on the accumulated gradient scaled by
// inv; clears the accumulator
__device__ __forceinline__ void adam_one(int k, float *theta, float *m, float *v, float *grad, float inv, float c1,
                                         float c2, float lr, float beta1, float beta2, float eps) {
  const float g = __ldcg(grad + k) * inv;   // summed by the training kernel's atomics (in L2)
  const float mk = beta1 * m[k] + (1.f - beta1) * g;
  const float vk = beta2 * v[k] + (1.f - beta2) * g * g;
  m[k] = mk;
  v[k] = vk;
  theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  grad[k] = 0.f;
}

// dynamic shared memory layout of k_mlp_train (bytes)
constexpr int TR_SMEM = (int)sizeof(MlpDev) + 2 * (TR_ROWS * MLP_IN + 4 * TR_ROWS * MLP_H + TR_ROWS * MLP_OUTP) +
                        4 * (TR_ROWS * MLP_OUT + MLP_NPARAM);

__global__ void __launch_bounds__(TR_ROWS * 2) k_mlp_train(TrainArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  MlpDev &w = *reinterpret_cast<MlpDev *>(smem);
  __nv_bfloat16 *sX = reinterpret_cast<__nv_bfloat16 *>(smem + sizeof(MlpDev));
  __nv_bfloat16 *sH1 = sX + TR_ROWS * MLP_IN;
  __nv_bfloat16 *sH2 = sH1 + TR_ROWS * MLP_H;
  __nv_bfloat16 *sD2 = sH2 + TR_ROWS * MLP_H;    // dL/da2
  __nv_bfloat16 *sD1 = sD2 + TR_ROWS * MLP_H;    // dL/da1
  __nv_bfloat16 *sDz = sD1 + TR_ROWS * MLP_H;    // dL/dz, padded to 16 columns
  float *sZ = reinterpret_cast<float *>(sDz + TR_ROWS * MLP_OUTP);
  float *sG = sZ + TR_ROWS * MLP_OUT;
  const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5;
  const int r0 = blockIdx.x * TR_ROWS;
  // model + rows
  {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(a.model);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&w);
    for (int k = tid; k < (int)(sizeof(MlpDev) / 4); k += nth) dst[k] = src[k];
  }
  for (int k = tid; k < TR_ROWS * MLP_IN; k += nth) {
    const int r = k / MLP_IN, c = k % MLP_IN;
    sX[k] = r0 + r < a.batch ? a.X[(size_t)a.idx[r0 + r] * MLP_IN + c] : __float2bfloat16_rn(0.f);
  }
  for (int k = tid; k < MLP_NPARAM; k += nth) sG[k] = 0.f;
  __syncthreads();
  // forward: warps 0..3 each take one 16-row tile
  if (warp < TR_WARPS) {
    const int m0 = warp * 16;
    mlp_forward_tile(w, sX + m0 * MLP_IN, sH1 + m0 * MLP_H, sH2 + m0 * MLP_H,
                     [&](int m, int n, float v) { sZ[(m0 + m) * MLP_OUT + n] = v; });
  }
  __syncthreads();
  // softmax cross-entropy gradient (weighted, not yet normalised by the batch weight)
  if (tid < TR_ROWS) {
    const int r = r0 + tid;
    float d[MLP_OUT] = {0.f, 0.f, 0.f};
    if (r < a.batch) {
      const int yy = a.y[a.idx[r]];
      const float cw = a.cw[yy];
      const float z0 = sZ[tid * 3], z1 = sZ[tid * 3 + 1], z2 = sZ[tid * 3 + 2];
      const float mx = fmaxf(z0, fmaxf(z1, z2));
      const float e0 = __expf(z0 - mx), e1 = __expf(z1 - mx), e2 = __expf(z2 - mx);
      const float s = e0 + e1 + e2;
      d[0] = cw * (e0 / s - (yy == 0));
      d[1] = cw * (e1 / s - (yy == 1));
      d[2] = cw * (e2 / s - (yy == 2));
      const float zy = yy == 0 ? z0 : (yy == 1 ? z1 : z2);
      atomicAdd(&a.stats[0], cw);
      atomicAdd(&a.stats[1], cw * (logf(s) + mx - zy));
    }
    for (int n = 0; n < MLP_OUTP; ++n) sDz[tid * MLP_OUTP + n] = __float2bfloat16_rn(n < MLP_OUT ? d[n] : 0.f);
    for (int n = 0; n < MLP_OUT; ++n) atomicAdd(&sG[OFF_B3 + n], d[n]);
  }
  __syncthreads();
  // backward data: da2 = (dz W3) * [h2 > 0]; da1 = (da2 W2) * [h1 > 0]
  if (warp < TR_WARPS) {
    const int m0 = warp * 16;
    uint32_t af[4], bf[2];
    load_a(af, [&](int m, int k) { return sDz[(m0 + m) * MLP_OUTP + k]; });
#pragma unroll
    for (int nt = 0; nt < MLP_H / 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      load_b(bf, [&](int k, int n) { return w.w3[k * MLP_H + nt * 8 + n]; });
      mma16816(c, af, bf);
      store_c(c, [&](int m, int n, float v) {
        const int o = (m0 + m) * MLP_H + nt * 8 + n;
        sD2[o] = __float2bfloat16_rn(__bfloat162float(sH2[o]) > 0.f ? v : 0.f);
      });
    }
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < MLP_H / 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < MLP_H / 16; ++ks) {
        load_a(af, [&](int m, int k) { return sD2[(m0 + m) * MLP_H + ks * 16 + k]; });
        load_b(bf, [&](int k, int n) { return w.w2[(ks * 16 + k) * MLP_H + nt * 8 + n]; });
        mma16816(c, af, bf);
      }
      store_c(c, [&](int m, int n, float v) {
        const int o = (m0 + m) * MLP_H + nt * 8 + n;
        sD1[o] = __float2bfloat16_rn(__bfloat162float(sH1[o]) > 0.f ? v : 0.f);
      });
    }
  }
  __syncthreads();
  // weight gradients over this block's rows (K = TR_ROWS): dW = dA^T H
  // tiles: dW2 4x8, dW1 4x2, dW3 1x8 (output rows padded to 16)
  for (int tile = warp; tile < 32 + 8 + 8; tile += nth / 32) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t af[4], bf[2];
    if (tile < 32) {   // dW2[o][i] = sum_r da2[r][o] h1[r][i]
      const int mt = tile / 8, nt = tile % 8;
#pragma unroll
      for (int ks = 0; ks < TR_ROWS / 16; ++ks) {
        load_a(af, [&](int m, int k) { return sD2[(ks * 16 + k) * MLP_H + mt * 16 + m]; });
        load_b(bf, [&](int k, int n) { return sH1[(ks * 16 + k) * MLP_H + nt * 8 + n]; });
        mma16816(c, af, bf);
      }
      store_c(c, [&](int m, int n, float v) { sG[OFF_W2 + (mt * 16 + m) * MLP_H + nt * 8 + n] += v; });
    } else if (tile < 40) {   // dW1[o][i] = sum_r da1[r][o] x[r][i]
      const int mt = (tile - 32) / 2, nt = (tile - 32) % 2;
#pragma unroll
      for (int ks = 0; ks < TR_ROWS / 16; ++ks) {
        load_a(af, [&](int m, int k) { return sD1[(ks * 16 + k) * MLP_H + mt * 16 + m]; });
        load_b(bf, [&](int k, int n) { return sX[(ks * 16 + k) * MLP_IN + nt * 8 + n]; });
        mma16816(c, af, bf);
      }
      store_c(c, [&](int m, int n, float v) { sG[OFF_W1 + (mt * 16 + m) * MLP_IN + nt * 8 + n] += v; });
    } else {   // dW3[o][i] = sum_r dz[r][o] h2[r][i]
      const int nt = tile - 40;
#pragma unroll
      for (int ks = 0; ks < TR_ROWS / 16; ++ks) {
        load_a(af, [&](int m, int k) { return sDz[(ks * 16 + k) * MLP_OUTP + m]; });
        load_b(bf, [&](int k, int n) { return sH2[(ks * 16 + k) * MLP_H + nt * 8 + n]; });
        mma16816(c, af, bf);
      }
      store_c(c, [&](int m, int n, float v) {
        if (m < MLP_OUT) sG[OFF_W3 + m * MLP_H + nt * 8 + n] += v;
      });
    }
  }
  // bias gradients: column sums of da1, da2
  for (int o = tid; o < 2 * MLP_H; o += nth) {
    const __nv_bfloat16 *D = o < MLP_H ? sD1 : sD2;
    const int col = o % MLP_H;
    float s = 0.f;
    for (int r = 0; r < TR_ROWS; ++r) s += __bfloat162float(D[r * MLP_H + col]);
    sG[(o < MLP_H ? OFF_B1 : OFF_B2) + col] += s;
  }
  __syncthreads();
  for (int k = tid; k < MLP_NPARAM; k += nth) atomicAdd(&a.grad[k], sG[k]);
}

// ------------------------------------------------------------------------------------
// training on the 5th-generation tensor core (tcgen05, accumulators in TMEM)
// ------------------------------------------------------------------------------------

// One CTA of four warps takes 128 samples; thread r owns sample r, whose accumulator rows
// sit in TMEM lane r (its warp's quarter).  Every product is one 128-row tcgen05.mma chain
// (BF16 operands in K-major canonical shared-memory tiles, FP32 accumulators in TMEM),
// issued by thread 0 and completed on one mbarrier:
//   forward      Z1 = X W1^T, Z2 = H1 W2^T, Z3 = H2 W3^T (W3 padded to 16 outputs);
//   backward     dH2 = dZ W3, dH1 = dA2 W2 (with transposed copies of W3 and W2);
//   weights      over the 128 samples (K = 128): [dA2^T ; dA1^T] [H1^T ; X^T ; 1]^T gives
//                dW2 (rows 0..63, columns 0..63), dW1 (rows 64..127, columns 64..79) and the
//                hidden bias gradients (column 80: the row of ones), and H2^T dZ gives dW3^T.
// The roundings are those of the mma.sync kernel: activations and hidden gradients to BF16
// where they enter a product, the output gradient to BF16 as an operand (its bias gradient
// from the FP32 values).  Rows that a product computes but nothing reads (padding) may
// hold any value.  Every wait is bounded; on a timeout the CTA records it in err, waits
// once more for its MMAs in flight, frees its TMEM and returns.
constexpr int TC_ROWS = 128;
constexpr int TC_COLS = 512;   // TMEM columns held (one CTA per SM: its shared memory)
constexpr unsigned TC_WAIT_LIMIT = 1u << 20;
// shared memory (byte offsets; K-major canonical tiles, rows x K)
constexpr int TC_X = 0;                          // X [128 x 16]
constexpr int TC_W1 = TC_X + 128 * 16 * 2;       // W1 [64 x 16]
constexpr int TC_W2 = TC_W1 + 64 * 16 * 2;       // W2 [64 x 64]
constexpr int TC_W2T = TC_W2 + 64 * 64 * 2;      // W2^T [64 x 64]
constexpr int TC_W3 = TC_W2T + 64 * 64 * 2;      // W3 padded [16 x 64]
constexpr int TC_W3T = TC_W3 + 16 * 64 * 2;      // (W3 padded)^T [64 x 16]
constexpr int TC_H1 = TC_W3T + 64 * 16 * 2;      // H1 [128 x 64]
constexpr int TC_H2 = TC_H1 + 128 * 64 * 2;      // H2 [128 x 64]
constexpr int TC_DZ = TC_H2 + 128 * 64 * 2;      // dZ padded [128 x 16]
constexpr int TC_DA2 = TC_DZ + 128 * 16 * 2;     // dA2 [128 x 64]
constexpr int TC_GAA = TC_DA2 + 128 * 64 * 2;    // [dA2^T ; dA1^T] [128 x 128]
constexpr int TC_GAB = TC_GAA + 128 * 128 * 2;   // [H1^T ; X^T ; ones ; unused] [96 x 128]
constexpr int TC_GBA = TC_GAB + 96 * 128 * 2;    // [H2^T ; unused] [128 x 128]
constexpr int TC_GBB = TC_GBA + 128 * 128 * 2;   // dZ^T padded [16 x 128]
constexpr int TC_BIAS = TC_GBB + 16 * 128 * 2;   // b1 [64], b2 [64], b3 [16] (FP32)
constexpr int TC_MISC = TC_BIAS + (64 + 64 + 16) * 4;   // mbarrier, TMEM base, block sums
constexpr int TC_SMEM = TC_MISC + 64;
// TMEM columns of the accumulators
constexpr int TM_Z1 = 0, TM_Z2 = 64, TM_Z3 = 128, TM_DH2 = 160, TM_DH1 = 224, TM_GA = 288, TM_GB = 384;
static_assert(TM_GB + 16 <= TC_COLS, "TMEM columns");

// 16 FP32 values -> 16 BF16 in two 16-byte words (elements 0..7, 8..15)
__device__ __forceinline__ void pack16_bf16(const float v[16], uint4 &lo, uint4 &hi) {
  lo = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
  hi = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]), pack_bf16(v[14], v[15]));
}

__global__ void __launch_bounds__(TC_ROWS) k_mlp_train_tc(TrainArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, r = tid;
  const int row = blockIdx.x * TC_ROWS + r;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + TC_MISC);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + TC_MISC + 8);
  float *sums = reinterpret_cast<float *>(sm + TC_MISC + 16);   // dZ column sums (3), weight, loss
  float *bias = reinterpret_cast<float *>(sm + TC_BIAS);
  const uint32_t s0 = smem_u32(sm);
  auto bfp = [&](int off) { return reinterpret_cast<__nv_bfloat16 *>(sm + off); };
  auto u4p = [&](int off) { return reinterpret_cast<uint4 *>(sm + off); };
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (tid < 5) sums[tid] = 0.f;
  if (warp == 0) tmem_alloc(tslot, TC_COLS);
  // the model's BF16 operands (and transposed copies) and FP32 biases, packed from the FP32
  // parameters as k_mlp_pack packs them: every 16-byte word of the parameter vector loaded
  // at once (one round trip), then each element placed in its tiles
  {
    static_assert(OFF_W2 % 4 == 0 && OFF_B2 % 4 == 0 && OFF_W3 % 4 == 0 && OFF_B3 % 4 == 0, "16-byte words");
    constexpr int NW = OFF_B3 / 4;                              // words before b3 (b3: 3 floats)
    constexpr int PER = (NW + TC_ROWS - 1) / TC_ROWS;
    const float4 *t4 = reinterpret_cast<const float4 *>(a.theta);
    float4 w4[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int q = tid + j * TC_ROWS;
      w4[j] = q < NW ? t4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    auto place = [&](int e, float x) {
      if (e < OFF_B1) {
        *bfp(TC_W1 + kmaj_off(e / MLP_IN, e % MLP_IN, MLP_IN)) = __float2bfloat16_rn(x);
      } else if (e < OFF_W2) {
        bias[e - OFF_B1] = x;
      } else if (e < OFF_B2) {
        const int o = (e - OFF_W2) / MLP_H, k = (e - OFF_W2) % MLP_H;
        const __nv_bfloat16 w = __float2bfloat16_rn(x);
        *bfp(TC_W2 + kmaj_off(o, k, MLP_H)) = w;
        *bfp(TC_W2T + kmaj_off(k, o, MLP_H)) = w;
      } else if (e < OFF_W3) {
        bias[MLP_H + e - OFF_B2] = x;
      } else {
        const int c = (e - OFF_W3) / MLP_H, k = (e - OFF_W3) % MLP_H;
        const __nv_bfloat16 w = __float2bfloat16_rn(x);
        *bfp(TC_W3 + kmaj_off(c, k, MLP_H)) = w;
        *bfp(TC_W3T + kmaj_off(k, c, MLP_OUTP)) = w;
      }
    };
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int q = tid + j * TC_ROWS;
      if (q < NW) {
        place(4 * q, w4[j].x);
        place(4 * q + 1, w4[j].y);
        place(4 * q + 2, w4[j].z);
        place(4 * q + 3, w4[j].w);
      }
    }
    // W3's padding rows (outputs 3..15) and b3 (3 values, then zeros)
    for (int e = tid; e < (MLP_OUTP - MLP_OUT) * MLP_H; e += TC_ROWS) {
      const int c = MLP_OUT + e / MLP_H, k = e % MLP_H;
      *bfp(TC_W3 + kmaj_off(c, k, MLP_H)) = __float2bfloat16_rn(0.f);
      *bfp(TC_W3T + kmaj_off(k, c, MLP_OUTP)) = __float2bfloat16_rn(0.f);
    }
    if (tid < MLP_OUTP) bias[2 * MLP_H + tid] = tid < MLP_OUT ? a.theta[OFF_B3 + tid] : 0.f;
  }
  // this thread's sample: features (two 16-byte words), label and class weight
  uint4 x0 = make_uint4(0, 0, 0, 0), x1 = x0;
  int yy = 0;
  float cw = 0.f;
  if (row < a.batch) {
    const int smp = a.idx[row];
    const uint4 *xp = reinterpret_cast<const uint4 *>(a.X + (size_t)smp * MLP_IN);
    x0 = xp[0];
    x1 = xp[1];
    yy = a.y[smp];
    cw = a.cw[yy];
  }
  *u4p(TC_X + kmaj_off(r, 0, MLP_IN)) = x0;
  *u4p(TC_X + kmaj_off(r, 8, MLP_IN)) = x1;
  {
    const __nv_bfloat16 *xa = reinterpret_cast<const __nv_bfloat16 *>(&x0);
    const __nv_bfloat16 *xb = reinterpret_cast<const __nv_bfloat16 *>(&x1);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      *bfp(TC_GAB + kmaj_off(64 + j, r, TC_ROWS)) = xa[j];
      *bfp(TC_GAB + kmaj_off(72 + j, r, TC_ROWS)) = xb[j];
    }
    *bfp(TC_GAB + kmaj_off(80, r, TC_ROWS)) = __float2bfloat16_rn(1.f);
  }

  uint32_t tm = 0;      // TMEM base (read after the first barrier)
  unsigned phase = 0;   // completions of the barrier so far
  // operands written -> one chain of MMAs -> its accumulators readable; false on a timeout
  // (the same answer in every thread)
  auto stage = [&](auto issue) -> bool {
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tm = *tslot;
    if (tid == 0 && !a.withhold) {
      issue(tm);
      umma_commit(bar);
    }
    __syncwarp();
    const unsigned limit = a.withhold ? 4096u : TC_WAIT_LIMIT;
    const bool done = mbar_wait(bar, phase & 1u, limit);
    tc_fence_after();
    if (__syncthreads_or(!done)) {
      if (tid == 0) atomicOr(a.err, 1u);
      mbar_wait(bar, phase & 1u, limit);   // the MMAs in flight, once more
      return false;
    }
    ++phase;
    return true;
  };
  auto finish = [&]() {
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tm, TC_COLS);
  };
  const uint32_t lane = (uint32_t)(warp * 32) << 16;   // this warp's TMEM lanes
  const uint32_t I64 = idesc_bf16_f32(128, 64), I16 = idesc_bf16_f32(128, 16), I96 = idesc_bf16_f32(128, 96);
  float v[16];
  uint4 lo, hi;

  // layer 1
  if (!stage([&](uint32_t t) {
        umma_bf16(t + TM_Z1, kmaj_desc(s0 + TC_X, MLP_IN), kmaj_desc(s0 + TC_W1, MLP_IN), I64, 0);
      })) {
    finish();
    return;
  }
  uint64_t mask1 = 0, mask2 = 0;   // ReLU masks of the BF16 activations
  for (int c = 0; c < MLP_H; c += 16) {
    tmem_ld16(tm + lane + TM_Z1 + c, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      v[q] = __bfloat162float(__float2bfloat16_rn(fmaxf(v[q] + bias[c + q], 0.f)));
      if (v[q] > 0.f) mask1 |= 1ull << (c + q);
      *bfp(TC_GAB + kmaj_off(c + q, r, TC_ROWS)) = __float2bfloat16_rn(v[q]);
    }
    pack16_bf16(v, lo, hi);
    *u4p(TC_H1 + kmaj_off(r, c, MLP_H)) = lo;
    *u4p(TC_H1 + kmaj_off(r, c + 8, MLP_H)) = hi;
  }
  // layer 2
  if (!stage([&](uint32_t t) {
        for (int ks = 0; ks < MLP_H / 16; ++ks)
          umma_bf16(t + TM_Z2, kmaj_desc(s0 + TC_H1 + 256 * ks, MLP_H), kmaj_desc(s0 + TC_W2 + 256 * ks, MLP_H), I64,
                    ks);
      })) {
    finish();
    return;
  }
  for (int c = 0; c < MLP_H; c += 16) {
    tmem_ld16(tm + lane + TM_Z2 + c, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      v[q] = __bfloat162float(__float2bfloat16_rn(fmaxf(v[q] + bias[MLP_H + c + q], 0.f)));
      if (v[q] > 0.f) mask2 |= 1ull << (c + q);
      *bfp(TC_GBA + kmaj_off(c + q, r, TC_ROWS)) = __float2bfloat16_rn(v[q]);
    }
    pack16_bf16(v, lo, hi);
    *u4p(TC_H2 + kmaj_off(r, c, MLP_H)) = lo;
    *u4p(TC_H2 + kmaj_off(r, c + 8, MLP_H)) = hi;
  }
  // layer 3, softmax cross-entropy gradient (class-weighted, not yet normalised)
  if (!stage([&](uint32_t t) {
        for (int ks = 0; ks < MLP_H / 16; ++ks)
          umma_bf16(t + TM_Z3, kmaj_desc(s0 + TC_H2 + 256 * ks, MLP_H), kmaj_desc(s0 + TC_W3 + 256 * ks, MLP_H), I16,
                    ks);
      })) {
    finish();
    return;
  }
  tmem_ld16(tm + lane + TM_Z3, v);
  float d[MLP_OUT] = {0.f, 0.f, 0.f};
  float wsum = 0.f, lsum = 0.f;
  if (row < a.batch) {
    const float z0 = v[0] + bias[2 * MLP_H], z1 = v[1] + bias[2 * MLP_H + 1], z2 = v[2] + bias[2 * MLP_H + 2];
    const float mx = fmaxf(z0, fmaxf(z1, z2));
    const float e0 = __expf(z0 - mx), e1 = __expf(z1 - mx), e2 = __expf(z2 - mx);
    const float se = e0 + e1 + e2;
    d[0] = cw * (e0 / se - (yy == 0));
    d[1] = cw * (e1 / se - (yy == 1));
    d[2] = cw * (e2 / se - (yy == 2));
    const float zy = yy == 0 ? z0 : (yy == 1 ? z1 : z2);
    wsum = cw;
    lsum = cw * (logf(se) + mx - zy);
  }
  {
    float red[5] = {d[0], d[1], d[2], wsum, lsum};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      for (int o = 16; o > 0; o >>= 1) red[q] += __shfl_xor_sync(0xffffffffu, red[q], o);
      if ((tid & 31) == 0) atomicAdd(&sums[q], red[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    v[q] = q < MLP_OUT ? d[q] : 0.f;
    *bfp(TC_GBB + kmaj_off(q, r, TC_ROWS)) = __float2bfloat16_rn(v[q]);
  }
  pack16_bf16(v, lo, hi);
  *u4p(TC_DZ + kmaj_off(r, 0, MLP_OUTP)) = lo;
  *u4p(TC_DZ + kmaj_off(r, 8, MLP_OUTP)) = hi;
  // dH2 = dZ W3
  if (!stage([&](uint32_t t) {
        umma_bf16(t + TM_DH2, kmaj_desc(s0 + TC_DZ, MLP_OUTP), kmaj_desc(s0 + TC_W3T, MLP_OUTP), I64, 0);
      })) {
    finish();
    return;
  }
  for (int c = 0; c < MLP_H; c += 16) {
    tmem_ld16(tm + lane + TM_DH2 + c, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      v[q] = (mask2 >> (c + q)) & 1ull ? v[q] : 0.f;
      *bfp(TC_GAA + kmaj_off(c + q, r, TC_ROWS)) = __float2bfloat16_rn(v[q]);
    }
    pack16_bf16(v, lo, hi);
    *u4p(TC_DA2 + kmaj_off(r, c, MLP_H)) = lo;
    *u4p(TC_DA2 + kmaj_off(r, c + 8, MLP_H)) = hi;
  }
  // dH1 = dA2 W2
  if (!stage([&](uint32_t t) {
        for (int ks = 0; ks < MLP_H / 16; ++ks)
          umma_bf16(t + TM_DH1, kmaj_desc(s0 + TC_DA2 + 256 * ks, MLP_H), kmaj_desc(s0 + TC_W2T + 256 * ks, MLP_H),
                    I64, ks);
      })) {
    finish();
    return;
  }
  for (int c = 0; c < MLP_H; c += 16) {
    tmem_ld16(tm + lane + TM_DH1 + c, v);
#pragma unroll
    for (int q = 0; q < 16; ++q)
      *bfp(TC_GAA + kmaj_off(MLP_H + c + q, r, TC_ROWS)) =
          __float2bfloat16_rn((mask1 >> (c + q)) & 1ull ? v[q] : 0.f);
  }
  // weight and hidden-bias gradients over the 128 samples
  if (!stage([&](uint32_t t) {
        for (int ks = 0; ks < TC_ROWS / 16; ++ks)
          umma_bf16(t + TM_GA, kmaj_desc(s0 + TC_GAA + 256 * ks, TC_ROWS), kmaj_desc(s0 + TC_GAB + 256 * ks, TC_ROWS),
                    I96, ks);
        for (int ks = 0; ks < TC_ROWS / 16; ++ks)
          umma_bf16(t + TM_GB, kmaj_desc(s0 + TC_GBA + 256 * ks, TC_ROWS), kmaj_desc(s0 + TC_GBB + 256 * ks, TC_ROWS),
                    I16, ks);
      })) {
    finish();
    return;
  }
  if (warp < 2) {   // rows 0..63: dW2 row r, b2, dW3 column r
    for (int c = 0; c < MLP_H; c += 16) {
      tmem_ld16(tm + lane + TM_GA + c, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) atomicAdd(&a.grad[OFF_W2 + r * MLP_H + c + q], v[q]);
    }
    tmem_ld16(tm + lane + TM_GA + 80, v);
    atomicAdd(&a.grad[OFF_B2 + r], v[0]);
    tmem_ld16(tm + lane + TM_GB, v);
#pragma unroll
    for (int q = 0; q < MLP_OUT; ++q) atomicAdd(&a.grad[OFF_W3 + q * MLP_H + r], v[q]);
  } else {   // rows 64..127: dW1 row r - 64, b1
    const int o = r - MLP_H;
    tmem_ld16(tm + lane + TM_GA + 64, v);
#pragma unroll
    for (int q = 0; q < MLP_IN; ++q) atomicAdd(&a.grad[OFF_W1 + o * MLP_IN + q], v[q]);
    tmem_ld16(tm + lane + TM_GA + 80, v);
    atomicAdd(&a.grad[OFF_B1 + o], v[0]);
  }
  __syncthreads();
  if (tid < MLP_OUT) atomicAdd(&a.grad[OFF_B3 + tid], sums[tid]);
  if (tid == MLP_OUT) atomicAdd(&a.stats[0], sums[3]);
  if (tid == MLP_OUT + 1) atomicAdd(&a.stats[1], sums[4]);
  finish();
}

// FP32 master parameters -> BF16 operand model
__global__ void k_mlp_pack(const float *theta, MlpDev *m) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MLP_H * MLP_H + MLP_H * MLP_IN + MLP_OUTP * MLP_H + 2 * MLP_H + MLP_OUTP;
       k += gridDim.x * blockDim.x) {
    int q = k;
    if (q < MLP_H * MLP_IN) { m->w1[q] = __float2bfloat16_rn(theta[OFF_W1 + q]); continue; }
    q -= MLP_H * MLP_IN;
    if (q < MLP_H * MLP_H) { m->w2[q] = __float2bfloat16_rn(theta[OFF_W2 + q]); continue; }
    q -= MLP_H * MLP_H;
    if (q < MLP_OUTP * MLP_H) {
      const int r = q / MLP_H;
      m->w3[q] = __float2bfloat16_rn(r < MLP_OUT ? theta[OFF_W3 + q] : 0.f);
      continue;
    }
    q -= MLP_OUTP * MLP_H;
    if (q < MLP_H) { m->b1[q] = theta[OFF_B1 + q]; continue; }
    q -= MLP_H;
    if (q < MLP_H) { m->b2[q] = theta[OFF_B2 + q]; continue; }
    q -= MLP_H;
    m->b3[q] = q < MLP_OUT ? theta[OFF_B3 + q] : 0.f;
  }
}

// Adam (Kingma & Ba 2015) on the normalised gradient; clears the accumulators
__global__ void k_mlp_adam(float *theta, float *m, float *v, float *grad, float *stats, int t, float lr,
                           float beta1, float beta2, float eps) {
  const float inv = stats[0] > 0.f ? 1.f / stats[0] : 0.f;
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MLP_NPARAM; k += gridDim.x * blockDim.x)
    adam_one(k, theta, m, v, grad, inv, c1, c2, lr, beta1, beta2, eps);
}

// Normalised copy of the accumulated gradient (divided by the batch's total class weight)
__global__ void k_mlp_scale(const float *grad, const float *stats, float *out) {
  const float inv = stats[0] > 0.f ? 1.f / stats[0] : 0.f;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MLP_NPARAM; k += gridDim.x * blockDim.x)
    out[k] = grad[k] * inv;
}

// Predictions (class, softmax margin top1 - top2, optionally the logits) for n samples; 4 warps
// x 16 rows per block
__global__ void __launch_bounds__(128) k_mlp_predict(const __nv_bfloat16 *X, int n, const MlpDev *model,
                                                     int *cls, float *margin, float *logits) {
  __shared__ MlpDev w;
  __shared__ __align__(16) __nv_bfloat16 sX[64 * MLP_IN];
  __shared__ __align__(16) __nv_bfloat16 sH1[64 * MLP_H];
  __shared__ float sZ[64 * MLP_OUT];
  const int tid = threadIdx.x, warp = tid >> 5;
  {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(model);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&w);
    for (int k = tid; k < (int)(sizeof(MlpDev) / 4); k += 128) dst[k] = src[k];
  }
  for (int r0 = blockIdx.x * 64; r0 < n; r0 += gridDim.x * 64) {
    __syncthreads();
    for (int k = tid; k < 64 * MLP_IN; k += 128) {
      const int r = k / MLP_IN;
      sX[k] = r0 + r < n ? X[(size_t)(r0 + r) * MLP_IN + k % MLP_IN] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    const int m0 = warp * 16;
    mlp_forward_tile(w, sX + m0 * MLP_IN, sH1 + m0 * MLP_H, nullptr,
                     [&](int m, int q, float v) { sZ[(m0 + m) * MLP_OUT + q] = v; });
    __syncthreads();
    if (tid < 64 && r0 + tid < n) {
      const float z0 = sZ[tid * 3], z1 = sZ[tid * 3 + 1], z2 = sZ[tid * 3 + 2];
      const float mx = fmaxf(z0, fmaxf(z1, z2));
      const float e0 = __expf(z0 - mx), e1 = __expf(z1 - mx), e2 = __expf(z2 - mx);
      const float s = e0 + e1 + e2;
      const float p0 = e0 / s, p1 = e1 / s, p2 = e2 / s;
      int c = 0;
      float top = p0, sec = fmaxf(p1, p2);
      if (p1 > top) { c = 1; sec = fmaxf(p0, p2); top = p1; }
      if (p2 > top) { c = 2; sec = fmaxf(p0, p1); top = p2; }
      cls[r0 + tid] = c;
      margin[r0 + tid] = top - sec;
      if (logits) {
        logits[(size_t)(r0 + tid) * 3] = z0;
        logits[(size_t)(r0 + tid) * 3 + 1] = z1;
        logits[(size_t)(r0 + tid) * 3 + 2] = z2;
      }
    }
  }
}

}  // namespace moss
