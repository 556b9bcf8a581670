// Learned importance-sampling proposal: a small MLP trained on the method's
// own (initial condition -> outcome) data, turned into a defensive-mixture
// proposal over (b^2, cos theta, phi, eta, chi) whose likelihood-ratio
// weights keep the cross-section estimator unbiased (every sampled
// trajectory is still integrated exactly).
//
// Tensor-core design (sm_103a, warp-level mma.sync m16n8k16, BF16 inputs,
// FP32 accumulation): each warp carries 16 samples through the network.  The
// accumulator fragment of two adjacent 16x8 output tiles has exactly the
// register layout of the A operand of a 16x16 slice, so a layer's SiLU output
// is fed to the next layer's products without touching shared memory.  The
// backward pass reuses the same fragments: dA = dZ W uses transposed weights
// staged in shared memory.  Training leaves each block round's transposed
// activations and errors in shared tiles; the weight gradients dW = dZ^T A
// are then block GEMMs over the round's samples (K = 128), accumulated in
// registers and added to the global gradient once per round.
//
// The network is ~9k multiply-adds per sample: negligible next to the
// trajectory integration, so a warp-level mma kernel is enough here.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "qcams.h"
#include "qcams_device.cuh"

namespace qcams {
namespace {

constexpr int IN = 8, H = 64, OUT = 4, NP = QCAMS_MLP_NPARAMS;
constexpr int OW1 = 0, OB1 = OW1 + H * IN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + H * H, OW4 = OB3 + H, OB4 = OW4 + OUT * H;
static_assert(OB4 + OUT == NP, "parameter layout");
static_assert(OW1 % 2 == 0 && OW2 % 2 == 0 && OW3 % 2 == 0 && OW4 % 2 == 0 && IN % 2 == 0,
              "weight-gradient pairs are 8-byte aligned");
constexpr int WARPS = 4, THREADS = WARPS * 32;
constexpr double kPi = 3.14159265358979323846;

struct Std {
  float mean[8], inv_std[8];
};

// Shared-memory weight tiles (BF16).  Forward B operands use W as [N][K];
// backward dA = dZ W needs W^T as [K][N].  Padding: W1 K 8 -> 16, W4 N 4 -> 8
// (forward) and W4^T N 4 -> 16.  Every row is padded by 8 elements (16 B):
// a fragment load touches rows g = 0..7 at words 2q / 2 + const, and the
// 16-byte row skew puts the 8 rows x 4 words on 32 distinct banks.
constexpr int PK = 8;   // row padding (BF16 elements)
struct alignas(16) WeightsSmem {   // 16-byte row-segment stores
  __nv_bfloat16 w1[H][16 + PK];
  __nv_bfloat16 w2[H][H + PK];
  __nv_bfloat16 w3[H][H + PK];
  __nv_bfloat16 w4[8][H + PK];
  __nv_bfloat16 w2t[H][H + PK];
  __nv_bfloat16 w3t[H][H + PK];
  __nv_bfloat16 w4t[H][16 + PK];
  float b1[H], b2[H], b3[H], b4[8];
};
// Training works in block rounds of RS = 64 CPW samples (4 warps x CPW
// chunks of 16).  Each chunk's forward and backward pass leave, in
// block-wide shared tiles, the transposed inputs, activations and
// back-propagated errors of its 16 samples (BF16, [unit][sample]); after the
// round each warp forms 16 rows of every weight gradient dW = dZ^T A as an
// MMA product over the round's samples, accumulated in registers and added
// to the global gradient once.  Rows are padded by 8 elements: a fragment
// load touches rows g = 0..7 at words q + const, and a row stride of
// 32 CPW + 4 words puts them on 32 distinct banks.
template <int CPW>
struct BlockTiles {
  static constexpr int RS = 16 * WARPS * CPW;   // samples per block round
  static constexpr int LDT = RS + PK;           // row stride (BF16 elements)
  __nv_bfloat16 xt[16][LDT];         // X^T  [feature (padded to 16)][sample]
  __nv_bfloat16 at[3][H][LDT];       // A1^T, A2^T, A3^T [unit][sample]
  __nv_bfloat16 dzt[3][H][LDT];      // dZ1^T, dZ2^T, dZ3^T [unit][sample]
  __nv_bfloat16 dz4t[16][LDT];       // dZ4^T [output (padded to 16)][sample]
};
// SiLU'(Z) of the warp's current chunk (layers 1-3), fragment order
// [i][lane], computed in the forward pass for the backward pass.
struct WarpZ {
  float ds[3][32][32];
};
// Bias gradients of the block (b1, b2, b3, b4), FP32 sums of the FP32 dZ
// fragments.
constexpr int GB1 = 0, NGB = 3 * H + OUT;
template <int CPW>
struct TrainSmem {
  WeightsSmem w;
  float gb[NGB];
  BlockTiles<CPW> t;
  WarpZ wz[WARPS];
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// D += A B for one m16n8k16 tile (BF16 in, FP32 accumulate).
__device__ __forceinline__ void mma(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Logistic function: __expf and the fast divide (a few ulp; the products it
// feeds are rounded to BF16).  For z below about -87 the quotient is 0.
__device__ __forceinline__ float sigm(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }

__device__ __forceinline__ __nv_bfloat16 bf_lo(uint32_t w) {
  return __ushort_as_bfloat16((unsigned short)(w & 0xffffu));
}
__device__ __forceinline__ __nv_bfloat16 bf_hi(uint32_t w) {
  return __ushort_as_bfloat16((unsigned short)(w >> 16));
}

// Weights to shared memory (blockDim.x == THREADS).  With p 16-byte aligned
// every matrix starts on a 16-byte boundary: each thread issues all of its
// 16-byte loads of 8-element row segments first, then stores each segment
// to its W row and, element by element, to the W^T column.  Otherwise,
// element loads.
__device__ void load_weights(WeightsSmem& W, const __nv_bfloat16* p, const float* pf) {
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
    constexpr int N1 = H * IN / 8, N2 = H * H / 8, N4 = OUT * H / 8;
    constexpr int NSEG = N1 + 2 * N2 + N4, PER = (NSEG + THREADS - 1) / THREADS;
    static_assert(IN == 8 && (OW2 % 8) == 0 && (OW3 % 8) == 0 && (OW4 % 8) == 0,
                  "16-byte row segments");
    uint4 v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = threadIdx.x + k * THREADS;
      int off = 0;
      if (i < N1) off = OW1 + 8 * i;
      else if (i < N1 + N2) off = OW2 + 8 * (i - N1);
      else if (i < N1 + 2 * N2) off = OW3 + 8 * (i - N1 - N2);
      else if (i < NSEG) off = OW4 + 8 * (i - N1 - 2 * N2);
      if (i < NSEG) v[k] = *reinterpret_cast<const uint4*>(p + off);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = threadIdx.x + k * THREADS;
      if (i >= NSEG) continue;
      const uint32_t w[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
      if (i < N1) {
        *reinterpret_cast<uint4*>(&W.w1[i][0]) = v[k];
        *reinterpret_cast<uint4*>(&W.w1[i][8]) = make_uint4(0u, 0u, 0u, 0u);
        continue;
      }
      const bool is4 = i >= N1 + 2 * N2;
      const int j = i < N1 + N2 ? i - N1 : i < N1 + 2 * N2 ? i - N1 - N2 : i - N1 - 2 * N2;
      const int r = j / (H / 8), c = 8 * (j % (H / 8));
      __nv_bfloat16* row = is4 ? &W.w4[r][c] : i < N1 + N2 ? &W.w2[r][c] : &W.w3[r][c];
      *reinterpret_cast<uint4*>(row) = v[k];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (is4) {
          W.w4t[c + 2 * e][r] = bf_lo(w[e]);
          W.w4t[c + 2 * e + 1][r] = bf_hi(w[e]);
        } else if (i < N1 + N2) {
          W.w2t[c + 2 * e][r] = bf_lo(w[e]);
          W.w2t[c + 2 * e + 1][r] = bf_hi(w[e]);
        } else {
          W.w3t[c + 2 * e][r] = bf_lo(w[e]);
          W.w3t[c + 2 * e + 1][r] = bf_hi(w[e]);
        }
      }
    }
    for (int i = threadIdx.x; i < (8 - OUT) * H; i += blockDim.x) W.w4[OUT + i / H][i % H] = zero;
    for (int i = threadIdx.x; i < H * (16 - OUT); i += blockDim.x)
      W.w4t[i / (16 - OUT)][OUT + i % (16 - OUT)] = zero;
  } else {
    for (int i = threadIdx.x; i < H * 16; i += blockDim.x) {
      const int r = i / 16, c = i % 16;
      W.w1[r][c] = c < IN ? p[OW1 + r * IN + c] : zero;
    }
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
      const int r = i / H, c = i % H;
      W.w2[r][c] = p[OW2 + i];
      W.w3[r][c] = p[OW3 + i];
      W.w2t[c][r] = p[OW2 + i];
      W.w3t[c][r] = p[OW3 + i];
    }
    for (int i = threadIdx.x; i < 8 * H; i += blockDim.x) {
      const int r = i / H, c = i % H;
      W.w4[r][c] = r < OUT ? p[OW4 + r * H + c] : zero;
    }
    for (int i = threadIdx.x; i < H * 16; i += blockDim.x) {
      const int r = i / 16, c = i % 16;
      W.w4t[r][c] = c < OUT ? p[OW4 + c * H + r] : zero;
    }
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    W.b1[i] = pf[OB1 + i];
    W.b2[i] = pf[OB2 + i];
    W.b3[i] = pf[OB3 + i];
  }
  if (threadIdx.x < 8) W.b4[threadIdx.x] = threadIdx.x < OUT ? pf[OB4 + threadIdx.x] : 0.0f;
}

// Features of the 16 rows handled by this lane's fragment rows: either from
// x[n][8] or (proposal mode) from the centre of grid cell `row`.
struct CellGrid {
  int n_b2, n_cth, n_phi, n_eta, n_chi;
  float E, v, j, b2_max;
};
__device__ __forceinline__ void features(const float* x, const int64_t* idx, int64_t n,
                                         int64_t row, const CellGrid* grid, float* f) {
  if (row >= n) {
    for (int k = 0; k < IN; ++k) f[k] = 0.0f;
    return;
  }
  if (!grid) {
    const int64_t r = idx ? idx[row] : row;   // minibatch rows gathered through idx
    for (int k = 0; k < IN; ++k) f[k] = x[r * IN + k];
    return;
  }
  int64_t c = row;
  const int i_chi = (int)(c % grid->n_chi); c /= grid->n_chi;
  const int i_eta = (int)(c % grid->n_eta); c /= grid->n_eta;
  const int i_phi = (int)(c % grid->n_phi); c /= grid->n_phi;
  const int i_cth = (int)(c % grid->n_cth); c /= grid->n_cth;
  const int i_b2 = (int)c;
  f[0] = grid->E;
  f[1] = sqrtf(grid->b2_max * (i_b2 + 0.5f) / grid->n_b2);
  f[2] = grid->v;
  f[3] = grid->j;
  f[4] = acosf(2.0f * (i_cth + 0.5f) / grid->n_cth - 1.0f);
  f[5] = 2.0f * (float)kPi * (i_phi + 0.5f) / grid->n_phi;
  f[6] = (i_chi + 0.5f) / grid->n_chi;
  f[7] = 2.0f * (float)kPi * (i_eta + 0.5f) / grid->n_eta;
}

// Forward pass of 16 samples (rows base .. base+15) by one warp.  Returns the
// logits fragment (rows g and g+8, columns 2q, 2q+1 of the padded 16x8 tile).
// With TRAIN, pre-activations go to the warp's z tiles and the transposed
// inputs and activations to the block tiles T, at sample columns col ..
// col + 15, for the backward pass.
template <bool TRAIN, int CPW>
__device__ void forward16(const WeightsSmem& W, WarpZ* wz, BlockTiles<CPW>* T, int col, const float* x,
                          const int64_t* idx, int64_t n, int64_t base, const CellGrid* grid,
                          const Std& sd, float* logit) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  float f0[IN], f1[IN];
  features(x, idx, n, base + g, grid, f0);
  features(x, idx, n, base + g + 8, grid, f1);
  for (int k = 0; k < IN; ++k) {
    f0[k] = (f0[k] - sd.mean[k]) * sd.inv_std[k];
    f1[k] = (f1[k] - sd.mean[k]) * sd.inv_std[k];
    if (base + g >= n) f0[k] = 0.0f;
    if (base + g + 8 >= n) f1[k] = 0.0f;
  }
  uint32_t a[4][4];  // A fragments of the current layer input (up to 4 k-slices)
  a[0][0] = pack2(f0[2 * q], f0[2 * q + 1]);
  a[0][1] = pack2(f1[2 * q], f1[2 * q + 1]);
  a[0][2] = 0u;
  a[0][3] = 0u;
  if (TRAIN) {
    T->xt[2 * q][col + g] = __float2bfloat16(f0[2 * q]);
    T->xt[2 * q + 1][col + g] = __float2bfloat16(f0[2 * q + 1]);
    T->xt[2 * q][col + g + 8] = __float2bfloat16(f1[2 * q]);
    T->xt[2 * q + 1][col + g + 8] = __float2bfloat16(f1[2 * q + 1]);
  }
  float c[8][4];
  for (int layer = 0; layer < 3; ++layer) {
    const float* bias = layer == 0 ? W.b1 : layer == 1 ? W.b2 : W.b3;
    const int ks = layer == 0 ? 1 : 4;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      c[t][0] = c[t][2] = bias[8 * t + 2 * q];
      c[t][1] = c[t][3] = bias[8 * t + 2 * q + 1];
      for (int s = 0; s < ks; ++s) {
        const __nv_bfloat16* wr = layer == 0 ? &W.w1[8 * t + g][0]
                                  : layer == 1 ? &W.w2[8 * t + g][16 * s]
                                               : &W.w3[8 * t + g][16 * s];
        mma(c[t], a[s], ld2(wr + 2 * q), ld2(wr + 8 + 2 * q));
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      // SiLU of tiles 2s (units 16s + 2q, +1) and 2s + 1 (units 16s + 8 + 2q,
      // +1), rows g and g + 8; with TRAIN also SiLU'(z) = sg (1 + z (1 - sg))
      float v[8];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float z = c[2 * s + h][e], sg = sigm(z);
          v[4 * h + e] = z * sg;
          if (TRAIN) wz->ds[layer][4 * (2 * s + h) + e][lane] = sg * (1.0f + z * (1.0f - sg));
        }
      a[s][0] = pack2(v[0], v[1]);
      a[s][1] = pack2(v[2], v[3]);
      a[s][2] = pack2(v[4], v[5]);
      a[s][3] = pack2(v[6], v[7]);
      if (TRAIN) {
        __nv_bfloat16 (*at)[BlockTiles<CPW>::LDT] = T->at[layer];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int u = 16 * s + 8 * h + 2 * q;
          at[u][col + g] = __float2bfloat16(v[4 * h]);
          at[u + 1][col + g] = __float2bfloat16(v[4 * h + 1]);
          at[u][col + g + 8] = __float2bfloat16(v[4 * h + 2]);
          at[u + 1][col + g + 8] = __float2bfloat16(v[4 * h + 3]);
        }
      }
    }
  }
  logit[0] = logit[2] = W.b4[2 * q];
  logit[1] = logit[3] = W.b4[2 * q + 1];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const __nv_bfloat16* wr = &W.w4[g][16 * s];
    mma(logit, a[s], ld2(wr + 2 * q), ld2(wr + 8 + 2 * q));
  }
}

// Softmax over the 4 logits of one row held by lanes q = 0 (columns 0, 1)
// and q = 1 (columns 2, 3); returns this lane's two probabilities.
__device__ __forceinline__ void softmax_pair(float z0, float z1, float* p0, float* p1) {
  const float o0 = __shfl_xor_sync(0xffffffffu, z0, 1);
  const float o1 = __shfl_xor_sync(0xffffffffu, z1, 1);
  const float m = fmaxf(fmaxf(z0, z1), fmaxf(o0, o1));
  const float e0 = __expf(z0 - m), e1 = __expf(z1 - m);
  const float s = e0 + e1 + __expf(o0 - m) + __expf(o1 - m);
  *p0 = e0 / s;
  *p1 = e1 / s;
}

// One warp's 16 rows m0 .. m0+15 of dW = dZ^T A over the round's RS samples,
// for the n_tiles 8-column tiles from column n0: A operand from dZ^T (rows
// = output units, samples contiguous), B operand from A^T (rows = input
// units, samples contiguous: the col layout of B), FP32 accumulation in
// registers; added once to the global gradient gW (row-major, n_in columns)
// for rows < n_out and columns < n_in.
template <int LDT>
__device__ void block_dw(const __nv_bfloat16 (*dzt)[LDT], const __nv_bfloat16 (*at)[LDT], int m0,
                         int n0, int n_tiles, int n_out, int n_in, float* gW) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  float d[8][4];
#pragma unroll
  for (int t = 0; t < 8; ++t) d[t][0] = d[t][1] = d[t][2] = d[t][3] = 0.0f;
#pragma unroll 2
  for (int ks = 0; ks < (LDT - PK) / 16; ++ks) {
    uint32_t a[4];
    a[0] = ld2(&dzt[m0 + g][16 * ks + 2 * q]);
    a[1] = ld2(&dzt[m0 + g + 8][16 * ks + 2 * q]);
    a[2] = ld2(&dzt[m0 + g][16 * ks + 8 + 2 * q]);
    a[3] = ld2(&dzt[m0 + g + 8][16 * ks + 8 + 2 * q]);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (t < n_tiles) {
        const __nv_bfloat16* br = &at[n0 + 8 * t + g][16 * ks];
        mma(d[t], a, ld2(br + 2 * q), ld2(br + 8 + 2 * q));
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if (t >= n_tiles) continue;
    const int r0 = m0 + g, r1 = r0 + 8, c = n0 + 8 * t + 2 * q;
    // c and n_in are even and the parameter offsets are even: 8-byte
    // aligned pairs (vector atomics, sm_90 and later)
    if (c < n_in) {
      if (r0 < n_out) atomicAdd(reinterpret_cast<float2*>(&gW[r0 * n_in + c]), make_float2(d[t][0], d[t][1]));
      if (r1 < n_out) atomicAdd(reinterpret_cast<float2*>(&gW[r1 * n_in + c]), make_float2(d[t][2], d[t][3]));
    }
  }
}

// Write dZ (fragment layout: 16 samples x `tiles` 8-unit tiles) transposed
// into the block tile dst at sample columns col .. col + 15.
template <int LDT>
__device__ __forceinline__ void store_dz(__nv_bfloat16 (*dst)[LDT], int col, const float (*dz)[4],
                                         int tiles) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  for (int t = 0; t < tiles; ++t) {
    const int c0 = 8 * t + 2 * q;
    dst[c0][col + g] = __float2bfloat16(dz[t][0]);
    dst[c0 + 1][col + g] = __float2bfloat16(dz[t][1]);
    dst[c0][col + g + 8] = __float2bfloat16(dz[t][2]);
    dst[c0 + 1][col + g + 8] = __float2bfloat16(dz[t][3]);
  }
}

// Bias gradient: sum over the 16 samples of dZ columns.
__device__ __forceinline__ void accumulate_db(const float (*dz)[4], int tiles, int n_valid,
                                              float* gb) {
  const int lane = threadIdx.x & 31, q = lane & 3;
  for (int t = 0; t < tiles; ++t) {
    float s0 = dz[t][0] + dz[t][2], s1 = dz[t][1] + dz[t][3];
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    const int col = 8 * t + 2 * q;
    if (lane < 4 && col < n_valid) {
      atomicAdd(&gb[col], s0);
      if (col + 1 < n_valid) atomicAdd(&gb[col + 1], s1);
    }
  }
}

// Gradient of the mean cross-entropy over n rows; with idx, row r of the
// minibatch is sample idx[r] of (x, label).  Block rounds of RS samples: each
// warp carries its chunks of 16 through the forward and backward passes
// (activations and errors to the block tiles, bias gradients to shared FP32
// sums), then the four weight gradients of the round are formed as block
// GEMMs (warp w: rows 16w .. 16w+15 of dW1..dW3, columns 16w .. 16w+15 of
// dW4) and added to the global gradient.
template <int CPW>
__global__ void __launch_bounds__(THREADS) k_mlp_grad(const __nv_bfloat16* pb, const float* pf,
                                                      Std sd, const float* x,
                                                      const uint8_t* label, const int64_t* idx,
                                                      int64_t n, float* grad, float* loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem<CPW>& S = *reinterpret_cast<TrainSmem<CPW>*>(smem_raw);
  constexpr int RS = BlockTiles<CPW>::RS, LDT = BlockTiles<CPW>::LDT;
  load_weights(S.w, pb, pf);
  for (int i = threadIdx.x; i < NGB; i += blockDim.x) S.gb[i] = 0.0f;
  // padding rows of the X^T and dZ4^T tiles (never written by the passes)
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  for (int i = threadIdx.x; i < (16 - IN) * LDT; i += blockDim.x) S.t.xt[IN + i / LDT][i % LDT] = zero;
  for (int i = threadIdx.x; i < (16 - 8) * LDT; i += blockDim.x) S.t.dz4t[8 + i / LDT][i % LDT] = zero;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  WarpZ* wz = &S.wz[warp];
  const float inv_n = 1.0f / (float)n;
  float loss_acc = 0.0f;
  const int64_t rounds = (n + RS - 1) / RS;
  for (int64_t rnd = blockIdx.x; rnd < rounds; rnd += gridDim.x) {
    for (int c = 0; c < CPW; ++c) {
      const int col = 16 * (WARPS * c + warp);
      const int64_t base = rnd * RS + col;
      float lg[4];
      forward16<true, CPW>(S.w, wz, &S.t, col, x, idx, n, base, nullptr, sd, lg);
      // softmax cross-entropy and dZ4 = (p - onehot) / n; rows past n and
      // rows without a target have dZ4 = 0 and so add nothing below
      float dz4[1][4] = {{0.f, 0.f, 0.f, 0.f}};
      float p[4];
      softmax_pair(lg[0], lg[1], &p[0], &p[1]);
      softmax_pair(lg[2], lg[3], &p[2], &p[3]);
      if (q < 2) {
        const int64_t r0 = base + g, r1 = base + g + 8;
        int l0 = r0 < n ? (int)label[idx ? idx[r0] : r0] : -1;
        int l1 = r1 < n ? (int)label[idx ? idx[r1] : r1] : -1;
        if (l0 >= OUT) l0 = -1;   // AMBIG / FAIL lanes carry no target
        if (l1 >= OUT) l1 = -1;
        for (int e = 0; e < 2; ++e) {
          const int k = 2 * q + e;
          if (l0 >= 0) {
            dz4[0][e] = (p[e] - (k == l0 ? 1.0f : 0.0f)) * inv_n;
            if (k == l0) loss_acc -= __logf(fmaxf(p[e], 1e-30f)) * inv_n;
          }
          if (l1 >= 0) {
            dz4[0][2 + e] = (p[2 + e] - (k == l1 ? 1.0f : 0.0f)) * inv_n;
            if (k == l1) loss_acc -= __logf(fmaxf(p[2 + e], 1e-30f)) * inv_n;
          }
        }
      }
      store_dz(S.t.dz4t, col, dz4, 1);
      accumulate_db(dz4, 1, OUT, &S.gb[3 * H]);
      // dA3 = dZ4 W4: A operand from the dZ4 fragment (K padded 8 -> 16)
      uint32_t a[4][4];
      a[0][0] = pack2(dz4[0][0], dz4[0][1]);
      a[0][1] = pack2(dz4[0][2], dz4[0][3]);
      a[0][2] = 0u;
      a[0][3] = 0u;
      float dz[8][4];
      for (int layer = 2; layer >= 0; --layer) {
        const int ks = layer == 2 ? 1 : 4;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          dz[t][0] = dz[t][1] = dz[t][2] = dz[t][3] = 0.0f;
          for (int s = 0; s < ks; ++s) {
            const __nv_bfloat16* wr = layer == 2 ? &S.w.w4t[8 * t + g][0]
                                      : layer == 1 ? &S.w.w3t[8 * t + g][16 * s]
                                                   : &S.w.w2t[8 * t + g][16 * s];
            mma(dz[t], a[s], ld2(wr + 2 * q), ld2(wr + 8 + 2 * q));
          }
          // dZ = dA * SiLU'(Z)
#pragma unroll
          for (int e = 0; e < 4; ++e) dz[t][e] *= wz->ds[layer][4 * t + e][lane];
        }
        store_dz(S.t.dzt[layer], col, dz, 8);
        accumulate_db(dz, 8, H, &S.gb[GB1 + H * layer]);
        if (layer > 0) {
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            a[s][0] = pack2(dz[2 * s][0], dz[2 * s][1]);
            a[s][1] = pack2(dz[2 * s][2], dz[2 * s][3]);
            a[s][2] = pack2(dz[2 * s + 1][0], dz[2 * s + 1][1]);
            a[s][3] = pack2(dz[2 * s + 1][2], dz[2 * s + 1][3]);
          }
        }
      }
    }
    __syncthreads();   // the round's tiles are complete
    const int m0 = 16 * warp;
    block_dw(S.t.dzt[0], S.t.xt, m0, 0, 1, H, IN, grad + OW1);
    block_dw(S.t.dzt[1], S.t.at[0], m0, 0, 8, H, H, grad + OW2);
    block_dw(S.t.dzt[2], S.t.at[1], m0, 0, 8, H, H, grad + OW3);
    block_dw(S.t.dz4t, S.t.at[2], 0, m0, 2, OUT, H, grad + OW4);
    __syncthreads();   // tiles are rewritten by the next round
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
  if (lane == 0 && loss) atomicAdd(loss, loss_acc);
  for (int i = threadIdx.x; i < NGB; i += blockDim.x) {
    const int k = i < 3 * H ? (i / H == 0 ? OB1 : i / H == 1 ? OB2 : OB3) + i % H : OB4 + (i - 3 * H);
    if (S.gb[i] != 0.0f) atomicAdd(&grad[k], S.gb[i]);
  }
}

__global__ void __launch_bounds__(THREADS) k_mlp_infer(const __nv_bfloat16* pb, const float* pf,
                                                       Std sd, const float* x, int64_t n,
                                                       CellGrid grid, int use_grid,
                                                       float* probs, double* g_out,
                                                       double eps) {
  __shared__ WeightsSmem W;
  load_weights(W, pb, pf);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int64_t chunks = (n + 15) / 16;
  for (int64_t ch = (int64_t)blockIdx.x * WARPS + warp; ch < chunks;
       ch += (int64_t)gridDim.x * WARPS) {
    const int64_t base = ch * 16;
    float lg[4], p[4];
    forward16<false, 1>(W, nullptr, nullptr, 0, x, nullptr, n, base, use_grid ? &grid : nullptr, sd,
                     lg);
    softmax_pair(lg[0], lg[1], &p[0], &p[1]);
    softmax_pair(lg[2], lg[3], &p[2], &p[3]);
    const int64_t r0 = base + g, r1 = base + g + 8;
    if (probs && q < 2) {
      if (r0 < n) { probs[r0 * 4 + 2 * q] = p[0]; probs[r0 * 4 + 2 * q + 1] = p[1]; }
      if (r1 < n) { probs[r1 * 4 + 2 * q] = p[2]; probs[r1 * 4 + 2 * q + 1] = p[3]; }
    }
    if (g_out) {
      // p_R = P(R_AC) + P(R_BC): columns 1 (lane q = 0) and 2 (lane q = 1)
      const float mine0 = q == 0 ? p[1] : p[0], mine1 = q == 0 ? p[3] : p[2];
      const float other0 = __shfl_xor_sync(0xffffffffu, mine0, 1);
      const float other1 = __shfl_xor_sync(0xffffffffu, mine1, 1);
      if (q == 0) {
        if (r0 < n) g_out[r0] = sqrt(eps + (double)mine0 + (double)other0);
        if (r1 < n) g_out[r1] = sqrt(eps + (double)mine1 + (double)other1);
      }
    }
  }
}

__global__ void k_adam(float* p, float* m, float* v, const float* grad, __nv_bfloat16* pb,
                       float lr, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NP; i += gridDim.x * blockDim.x) {
    const float gr = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * gr;
    const float vi = 0.999f * v[i] + 0.001f * gr * gr;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    p[i] = pi;
    pb[i] = __float2bfloat16(pi);
  }
}

// Minibatch indices for training step `step`: idx[i] uniform on [0, n) from
// Philox4x32-10 with key = seed and counter (i, step_lo, step_hi, 4); the
// 64-bit word w1:w0 is mapped by the high half of w * n (bias <= n / 2^64).
__global__ void k_draw_idx(int64_t* idx, int batch, int64_t n, uint64_t seed, uint64_t step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  const uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)step, (uint32_t)(step >> 32), 4u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const unsigned long long u = ((unsigned long long)w.y << 32) | w.x;
  idx[i] = (int64_t)__umul64hi(u, (unsigned long long)n);
}

__global__ void k_mlp_init(float* p, float* m, float* v, __nv_bfloat16* pb, uint64_t seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NP; i += gridDim.x * blockDim.x) {
    float fan_in = 0.0f;
    if (i < OB1) fan_in = IN;
    else if (i >= OW2 && i < OB2) fan_in = H;
    else if (i >= OW3 && i < OB3) fan_in = H;
    else if (i >= OW4 && i < OB4) fan_in = H;
    float val = 0.0f;
    if (fan_in > 0.0f) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)i, 0u, 3u, 0u),
                                    make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
      const float u = (float)u01(w.x);
      val = (2.0f * u - 1.0f) * rsqrtf(fan_in);
    }
    p[i] = val;
    m[i] = 0.0f;
    v[i] = 0.0f;
    pb[i] = __float2bfloat16(val);
  }
}

__global__ void k_mlp_sync(const float* p, __nv_bfloat16* pb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NP; i += gridDim.x * blockDim.x)
    pb[i] = __float2bfloat16(p[i]);
}

__global__ void k_features(int64_t n, const double* E, const double* b, const int32_t* v,
                           const int32_t* j, const double* u0, const double* u1,
                           const double* u2, const double* u3, float* x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i * 8 + 0] = (float)E[i];
  x[i * 8 + 1] = (float)b[i];
  x[i * 8 + 2] = (float)v[i];
  x[i * 8 + 3] = (float)j[i];
  x[i * 8 + 4] = (float)acos(fmin(1.0, fmax(-1.0, 2.0 * u0[i] - 1.0)));
  x[i * 8 + 5] = (float)(2.0 * kPi * u1[i]);
  x[i * 8 + 6] = (float)u3[i];
  x[i * 8 + 7] = (float)(2.0 * kPi * u2[i]);
}

__global__ void k_moments(const float* x, int64_t n, double* acc) {
  __shared__ double s[16];
  if (threadIdx.x < 16) s[threadIdx.x] = 0.0;
  __syncthreads();
  double loc[16] = {0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < 8; ++k) {
      const double v = x[i * 8 + k];
      loc[k] += v;
      loc[8 + k] += v * v;
    }
  for (int k = 0; k < 16; ++k) atomicAdd(&s[k], loc[k]);
  __syncthreads();
  if (threadIdx.x < 16) atomicAdd(&acc[threadIdx.x], s[threadIdx.x]);
}

// Normalise the proposal and form its integer CDF in one block with a fixed
// summation order (deterministic bits).  g holds g_c on entry, q_c on exit.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_proposal_finish(double* g, int64_t n_cells,
                                                                  double alpha, int64_t* qfix,
                                                                  int64_t* cdf) {
  __shared__ double ds[kScanThreads];
  __shared__ long long ls[kScanThreads];
  const int t = threadIdx.x;
  const int64_t per = (n_cells + kScanThreads - 1) / kScanThreads;
  const int64_t lo = t * per, hi = min(n_cells, lo + per);
  double sum = 0.0;
  for (int64_t c = lo; c < hi; ++c) sum += g[c];
  ds[t] = sum;
  __syncthreads();
  for (int o = kScanThreads / 2; o > 0; o >>= 1) {
    if (t < o) ds[t] += ds[t + o];
    __syncthreads();
  }
  const double total = ds[0];
  long long part = 0;
  for (int64_t c = lo; c < hi; ++c) {
    const double qc = alpha / (double)n_cells + (1.0 - alpha) * g[c] / total;
    g[c] = qc;
    const long long qi = __double2ll_rn(qc * 1099511627776.0);  // 2^40
    qfix[c] = qi;
    part += qi;
  }
  ls[t] = part;
  __syncthreads();
  // inclusive scan of the per-thread parts (Hillis-Steele)
  for (int o = 1; o < kScanThreads; o <<= 1) {
    long long v = t >= o ? ls[t - o] : 0;
    __syncthreads();
    ls[t] += v;
    __syncthreads();
  }
  long long run = t > 0 ? ls[t - 1] : 0;
  for (int64_t c = lo; c < hi; ++c) {
    run += qfix[c];
    cdf[c] = run;
  }
}

__global__ void k_sample(CellGrid grid, int64_t n_cells, const int64_t* qfix, const int64_t* cdf,
                         int64_t n, uint64_t seed, uint64_t id_offset, double b2_max, double* b,
                         double* u0, double* u1, double* u2, double* u3, double* w,
                         int32_t* cell) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t id = id_offset + (uint64_t)i;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint4 wa = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), 1u, 0u), key);
  const uint4 wb = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), 2u, 0u), key);
  const unsigned long long total = (unsigned long long)cdf[n_cells - 1];
  // U = floor(u_0 total) with u_0 = (w + 1/2) 2^-32, in exact integer arithmetic:
  // (2 w + 1) total / 2^33
  const unsigned long long m = 2ull * wa.x + 1ull;
  const unsigned long long lo = m * total, hi = __umul64hi(m, total);
  const unsigned long long U = (hi << 31) | (lo >> 33);
  int64_t a = 0, z = n_cells - 1;
  while (a < z) {
    const int64_t mid = (a + z) >> 1;
    if ((unsigned long long)cdf[mid] > U) z = mid;
    else a = mid + 1;
  }
  int64_t c = a;
  cell[i] = (int32_t)c;
  const int i_chi = (int)(c % grid.n_chi); c /= grid.n_chi;
  const int i_eta = (int)(c % grid.n_eta); c /= grid.n_eta;
  const int i_phi = (int)(c % grid.n_phi); c /= grid.n_phi;
  const int i_cth = (int)(c % grid.n_cth); c /= grid.n_cth;
  const int i_b2 = (int)c;
  const double b2 = b2_max * (i_b2 + u01(wa.y)) / grid.n_b2;
  b[i] = sqrt(b2);
  u0[i] = (i_cth + u01(wa.z)) / grid.n_cth;
  u1[i] = (i_phi + u01(wa.w)) / grid.n_phi;
  u2[i] = (i_eta + u01(wb.x)) / grid.n_eta;
  u3[i] = (i_chi + u01(wb.y)) / grid.n_chi;
  w[i] = ((double)total / (double)n_cells) / (double)qfix[a];
}

int dev_ok() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QCAMS_E_NODEVICE;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
    return QCAMS_E_NODEVICE;
  return (major == 10 && minor == 3) ? QCAMS_OK : QCAMS_E_NODEVICE;
}

bool mlp_ok(const qcams_mlp* m) {
  return m && m->params && m->adam_m && m->adam_v && m->grad && m->params_bf16;
}

Std std_of(const qcams_mlp* m) {
  Std s;
  for (int k = 0; k < 8; ++k) {
    s.mean[k] = m->x_mean[k];
    s.inv_std[k] = m->x_std[k] > 0.f ? 1.0f / m->x_std[k] : 1.0f;
  }
  return s;
}

int sm_count() {
  int dev = 0, s = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
  return s > 0 ? s : 1;
}

int status_of(cudaError_t e) { return e == cudaSuccess ? QCAMS_OK : QCAMS_E_CUDA; }

// Proposal spec check: QCAMS_E_INVALID for bad fields, QCAMS_E_CAPACITY for
// more than 2^22 cells.
int grid_status(const qcams_proposal_spec* s) {
  if (!s || s->n_b2 < 1 || s->n_cth < 1 || s->n_phi < 1 || s->n_eta < 1 || s->n_chi < 1)
    return QCAMS_E_INVALID;
  if (!(s->b2_max > 0) || !(s->alpha > 0) || !(s->alpha <= 1) || !(s->eps >= 0) ||
      !std::isfinite(s->E_col))
    return QCAMS_E_INVALID;
  const double n = (double)s->n_b2 * s->n_cth * s->n_phi * s->n_eta * s->n_chi;
  return n <= (double)(1 << 22) ? QCAMS_OK : QCAMS_E_CAPACITY;
}

CellGrid grid_of(const qcams_proposal_spec* s) {
  CellGrid g;
  g.n_b2 = s->n_b2;
  g.n_cth = s->n_cth;
  g.n_phi = s->n_phi;
  g.n_eta = s->n_eta;
  g.n_chi = s->n_chi;
  g.E = (float)s->E_col;
  g.v = (float)s->v;
  g.j = (float)s->j;
  g.b2_max = (float)s->b2_max;
  return g;
}

template <int CPW>
cudaError_t launch_grad_cpw(const qcams_mlp* m, const float* x, const uint8_t* label,
                            const int64_t* idx, int64_t n, float* loss_out, cudaStream_t st) {
  const size_t smem = sizeof(TrainSmem<CPW>);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad<CPW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int64_t grid = (n + BlockTiles<CPW>::RS - 1) / BlockTiles<CPW>::RS;
  if (grid > sm_count()) grid = sm_count();
  if (grid < 1) grid = 1;
  k_mlp_grad<CPW><<<(unsigned)grid, THREADS, smem, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(m->params_bf16), m->params, std_of(m), x, label, idx,
      n, m->grad, loss_out);
  return cudaGetLastError();
}

int launch_grad(const qcams_mlp* m, const float* x, const uint8_t* label, const int64_t* idx,
                int64_t n, float* loss_out, bool zero_loss, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(m->grad, 0, NP * sizeof(float), st);
  if (e == cudaSuccess && loss_out && zero_loss) e = cudaMemsetAsync(loss_out, 0, sizeof(float), st);
  if (e != cudaSuccess) return QCAMS_E_CUDA;
  // At most one block per SM (the weights, the round's tiles and the warps'
  // SiLU' values take 155 KB of shared memory with 64-sample rounds, 203 KB
  // with 128).  A batch that fits one 64-sample round per SM (8,192 samples:
  // 128 blocks) takes that, the shortest block; larger batches take
  // 128-sample rounds, half the rounds' global-atomic flushes.
  e = (n + 63) / 64 <= sm_count() ? launch_grad_cpw<1>(m, x, label, idx, n, loss_out, st)
                                  : launch_grad_cpw<2>(m, x, label, idx, n, loss_out, st);
  return status_of(e);
}

int launch_adam(qcams_mlp* m, float lr, cudaStream_t st) {
  m->step += 1;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)m->step));
  const float c2 = (float)(1.0 - std::pow(0.999, (double)m->step));
  k_adam<<<36, 256, 0, st>>>(m->params, m->adam_m, m->adam_v, m->grad,
                             reinterpret_cast<__nv_bfloat16*>(m->params_bf16), lr, c1, c2);
  return status_of(cudaGetLastError());
}

}  // namespace
}  // namespace qcams

using namespace qcams;

extern "C" {

int qcams_mlp_init(qcams_mlp* m, uint64_t seed, void* cuda_stream) {
  if (!mlp_ok(m)) return QCAMS_E_INVALID;
  int rc;
  if ((rc = dev_ok()) != QCAMS_OK) return rc;
  for (int k = 0; k < 8; ++k) {
    m->x_mean[k] = 0.0f;
    m->x_std[k] = 1.0f;
  }
  m->step = 0;
  (void)cudaGetLastError();
  k_mlp_init<<<36, 256, 0, (cudaStream_t)cuda_stream>>>(
      m->params, m->adam_m, m->adam_v, reinterpret_cast<__nv_bfloat16*>(m->params_bf16), seed);
  return status_of(cudaGetLastError());
}

int qcams_mlp_sync(const qcams_mlp* m, void* cuda_stream) {
  if (!mlp_ok(m)) return QCAMS_E_INVALID;
  int rc;
  if ((rc = dev_ok()) != QCAMS_OK) return rc;
  (void)cudaGetLastError();
  k_mlp_sync<<<36, 256, 0, (cudaStream_t)cuda_stream>>>(
      m->params, reinterpret_cast<__nv_bfloat16*>(m->params_bf16));
  return status_of(cudaGetLastError());
}

int qcams_mlp_features(const qcams_batch* batch, const double* E_col, const double* b,
                       const int32_t* v, const int32_t* j, float* x, void* cuda_stream) {
  if (!batch || batch->n < 0) return QCAMS_E_INVALID;
  if (batch->n == 0) return QCAMS_OK;
  if (!E_col || !b || !v || !j || !x || !batch->u[0] || !batch->u[1] || !batch->u[2] ||
      !batch->u[3])
    return QCAMS_E_INVALID;
  int rc;
  if ((rc = dev_ok()) != QCAMS_OK) return rc;
  (void)cudaGetLastError();
  k_features<<<(unsigned)((batch->n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(
      batch->n, E_col, b, v, j, batch->u[0], batch->u[1], batch->u[2], batch->u[3], x);
  return status_of(cudaGetLastError());
}

int qcams_mlp_fit_standardizer(qcams_mlp* m, const float* x, int64_t n, void* cuda_stream) {
  if (!m || !x || n < 2) return QCAMS_E_INVALID;
  int rc;
  if ((rc = dev_ok()) != QCAMS_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* acc = nullptr;
  (void)cudaGetLastError();
  if (cudaMallocAsync((void**)&acc, 16 * sizeof(double), st) != cudaSuccess) return QCAMS_E_CUDA;
  cudaError_t e = cudaMemsetAsync(acc, 0, 16 * sizeof(double), st);
  if (e == cudaSuccess) {
    k_moments<<<sm_count() * 2, 256, 0, st>>>(x, n, acc);
    e = cudaGetLastError();
  }
  double h[16];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(acc, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return QCAMS_E_CUDA;
  for (int k = 0; k < 8; ++k) {
    const double mu = h[k] / (double)n;
    const double var = h[8 + k] / (double)n - mu * mu;
    m->x_mean[k] = (float)mu;
    m->x_std[k] = var > 1e-20 ? (float)std::sqrt(var) : 1.0f;
  }
  return QCAMS_OK;
}

int qcams_mlp_grad(const qcams_mlp* m, const float* x, const uint8_t* label, int64_t n,
                   float* loss_out, void* cuda_stream) {
  if (!mlp_ok(m) || !x || !label || n < 1) return QCAMS_E_INVALID;
  int rc;
  if ((rc = dev_ok()) != QCAMS_OK) return rc;
  (void)cudaGetLastError();
  return launch_grad(m, x, label, nullptr, n, loss_out, true, (cudaStream_t)cuda_stream);
}

int qcams_mlp_train_step(qcams_mlp* m, const float* x, const uint8_t* label, int64_t n,
                         float lr, float* loss_out, void* cuda_stream) {
  if (!(lr > 0.0f)) return QCAMS_E_INVALID;
  int rc = qcams_mlp_grad(m, x, label, n, loss_out, cuda_stream);
  if (rc != QCAMS_OK) return rc;
  return launch_adam(m, lr, (cudaStream_t)cuda_stream);
}

int qcams_mlp_train(qcams_mlp* m, const float* x, const uint8_t* label, int64_t n, int64_t steps,
                    int32_t batch, float lr, uint64_t seed, int64_t* idx, float* losses,
                    void* cuda_stream) {
  if (!mlp_ok(m) || !x || !label || !idx || n < 1 || steps < 0 || batch < 1 || !(lr > 0.0f))
    return QCAMS_E_INVALID;
  int rc;
  if ((rc = dev_ok()) != QCAMS_OK) return rc;
  (void)cudaGetLastError();
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (losses && steps > 0 &&
      cudaMemsetAsync(losses, 0, sizeof(float) * (size_t)steps, st) != cudaSuccess)
    return QCAMS_E_CUDA;
  for (int64_t s = 0; s < steps; ++s) {
    k_draw_idx<<<(batch + 255) / 256, 256, 0, st>>>(idx, batch, n, seed, (uint64_t)m->step);
    if (cudaGetLastError() != cudaSuccess) return QCAMS_E_CUDA;
    if ((rc = launch_grad(m, x, label, idx, batch, losses ? losses + s : nullptr, false, st)) !=
        QCAMS_OK)
      return rc;
    if ((rc = launch_adam(m, lr, st)) != QCAMS_OK) return rc;
  }
  return QCAMS_OK;
}

int qcams_mlp_infer(const qcams_mlp* m, const float* x, int64_t n, float* probs,
                    void* cuda_stream) {
  if (!mlp_ok(m) || !x || !probs || n < 0) return QCAMS_E_INVALID;
  if (n == 0) return QCAMS_OK;
  int rc;
  if ((rc = dev_ok()) != QCAMS_OK) return rc;
  (void)cudaGetLastError();
  const int64_t chunks = (n + 15) / 16;
  int64_t grid = (chunks + WARPS - 1) / WARPS;
  if (grid > 8 * sm_count()) grid = 8 * sm_count();
  CellGrid none{};
  k_mlp_infer<<<(unsigned)grid, THREADS, 0, (cudaStream_t)cuda_stream>>>(
      reinterpret_cast<const __nv_bfloat16*>(m->params_bf16), m->params, std_of(m), x, n, none,
      0, probs, nullptr, 0.0);
  return status_of(cudaGetLastError());
}

int qcams_build_proposal(const qcams_mlp* m, const qcams_proposal_spec* spec, double* q,
                         int64_t* qfix, int64_t* cdf, void* cuda_stream) {
  if (!mlp_ok(m) || !q || !qfix || !cdf) return QCAMS_E_INVALID;
  if (const int gs = grid_status(spec)) return gs;
  int rc;
  if ((rc = dev_ok()) != QCAMS_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t N = (int64_t)spec->n_b2 * spec->n_cth * spec->n_phi * spec->n_eta * spec->n_chi;
  const int64_t chunks = (N + 15) / 16;
  int64_t grid = (chunks + WARPS - 1) / WARPS;
  if (grid > 8 * sm_count()) grid = 8 * sm_count();
  (void)cudaGetLastError();
  k_mlp_infer<<<(unsigned)grid, THREADS, 0, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(m->params_bf16), m->params, std_of(m), nullptr, N,
      grid_of(spec), 1, nullptr, q, spec->eps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return QCAMS_E_CUDA;
  k_proposal_finish<<<1, kScanThreads, 0, st>>>(q, N, spec->alpha, qfix, cdf);
  return status_of(cudaGetLastError());
}

int qcams_sample_proposal(const qcams_proposal_spec* spec, const int64_t* qfix,
                          const int64_t* cdf, int64_t n, uint64_t seed, uint64_t id_offset,
                          double* b, double* const* u_out, double* w, int32_t* cell,
                          void* cuda_stream) {
  if (!qfix || !cdf || n < 0 || !b || !u_out || !w || !cell) return QCAMS_E_INVALID;
  if (const int gs = grid_status(spec)) return gs;
  if (!u_out[0] || !u_out[1] || !u_out[2] || !u_out[3]) return QCAMS_E_INVALID;
  if (n == 0) return QCAMS_OK;
  int rc;
  if ((rc = dev_ok()) != QCAMS_OK) return rc;
  const int64_t N = (int64_t)spec->n_b2 * spec->n_cth * spec->n_phi * spec->n_eta * spec->n_chi;
  (void)cudaGetLastError();
  k_sample<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(
      grid_of(spec), N, qfix, cdf, n, seed, id_offset, spec->b2_max, b, u_out[0], u_out[1],
      u_out[2], u_out[3], w, cell);
  return status_of(cudaGetLastError());
}

}  // extern "C"
