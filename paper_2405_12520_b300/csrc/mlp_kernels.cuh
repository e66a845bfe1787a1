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
};

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
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MLP_NPARAM; k += gridDim.x * blockDim.x) {
    const float g = grad[k] * inv;
    const float mk = beta1 * m[k] + (1.f - beta1) * g;
    const float vk = beta2 * v[k] + (1.f - beta2) * g * g;
    m[k] = mk;
    v[k] = vk;
    theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    grad[k] = 0.f;
  }
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
