// policy_train.cuh -- kernels of the learned-branching policy outside the
// search: feature extraction for training data, batched scoring, and one
// training step (forward, listwise softmax cross-entropy, backward, Adam).
// Every matrix product runs on the tensor cores through warp-level
// mma.sync m16n8k16 with BF16 operands and FP32 accumulation; the forward
// pass computes exactly what the search kernels compute (BF16 features,
// weights and first hidden layer, FP32 second layer and output).
#pragma once

#include <cuda_bf16.h>

#include "policy.cuh"

namespace pccp {

constexpr int kPolicyParams = 128 * 16 + 128 + 128 * 128 + 128 + 128 + 1;
// flat parameter layout (FP32 masters, gradients and Adam moments)
constexpr int kOffW1 = 0;                    // [128][16], inputs 12..15 stay 0
constexpr int kOffB1 = kOffW1 + 128 * 16;    // [128]
constexpr int kOffW2 = kOffB1 + 128;         // [128][128] (out, in)
constexpr int kOffB2 = kOffW2 + 128 * 128;   // [128]
constexpr int kOffW3 = kOffB2 + 128;         // [128]
constexpr int kOffB3 = kOffW3 + 128;         // [1]

__device__ __forceinline__ uint32_t pack_bf16_bits(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(lo)) |
         (static_cast<uint32_t>(__bfloat16_as_ushort(hi)) << 16);
}

// C[M x N] = op(A)[M x K] * op(B)[K x N]; BF16 in, FP32 out (row-major, ldc).
// op(A)(m, k) = TA ? A[k * lda + m] : A[m * lda + k]
// op(B)(k, n) = TB ? B[n * ldb + k] : B[k * ldb + n]
// M % 16 == 0, N % 8 == 0, K % 16 == 0; one warp per 16 x 8 output tile.
template <bool TA, bool TB>
__global__ void k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda,
                            const __nv_bfloat16* __restrict__ B, int ldb, float* __restrict__ C,
                            int ldc) {
  const int warp = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int tiles_n = N / 8;
  const int tm = warp / tiles_n, tn = warp - tm * tiles_n;
  if (tm * 16 >= M) return;  // whole warps leave together
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = tm * 16 + g, r1 = r0 + 8, n = tn * 8 + g;
  auto ea = [&](int m, int k) -> __nv_bfloat16 {
    return TA ? A[static_cast<size_t>(k) * lda + m] : A[static_cast<size_t>(m) * lda + k];
  };
  auto eb = [&](int k, int nn) -> __nv_bfloat16 {
    return TB ? B[static_cast<size_t>(nn) * ldb + k] : B[static_cast<size_t>(k) * ldb + nn];
  };
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int ka = k0 + 2 * t, kb = ka + 8;
    const uint32_t a[4] = {pack_bf16_bits(ea(r0, ka), ea(r0, ka + 1)),
                           pack_bf16_bits(ea(r1, ka), ea(r1, ka + 1)),
                           pack_bf16_bits(ea(r0, kb), ea(r0, kb + 1)),
                           pack_bf16_bits(ea(r1, kb), ea(r1, kb + 1))};
    const uint2 b = make_uint2(pack_bf16_bits(eb(ka, n), eb(ka + 1, n)),
                               pack_bf16_bits(eb(kb, n), eb(kb + 1, n)));
    mma_16816(acc, a, b);
  }
  const int c0 = tn * 8 + 2 * t;
  C[static_cast<size_t>(r0) * ldc + c0] = acc[0];
  C[static_cast<size_t>(r0) * ldc + c0 + 1] = acc[1];
  C[static_cast<size_t>(r1) * ldc + c0] = acc[2];
  C[static_cast<size_t>(r1) * ldc + c0 + 1] = acc[3];
}

// Features [n][12] FP32 -> BF16 rows of 16 (zero-padded), rows n..rows_pad-1 zero.
__global__ void k_pack_features(int n, int rows_pad, const float* __restrict__ f,
                                __nv_bfloat16* __restrict__ X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows_pad * 16) return;
  const int r = i >> 4, c = i & 15;
  const float v = (r < n && c < kPolicyFeatures) ? f[static_cast<size_t>(r) * kPolicyFeatures + c]
                                                  : 0.f;
  X[i] = __float2bfloat16_rn(v);
}

// H = relu(Z + b) (FP32) and its BF16 copy; Z, H: [rows][128].
__global__ void k_bias_relu(int rows, const float* __restrict__ Z, const float* __restrict__ b,
                            float* __restrict__ H, __nv_bfloat16* __restrict__ Hb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * 128) return;
  const float h = fmaxf(Z[i] + b[i & 127], 0.f);
  if (H) H[i] = h;
  if (Hb) Hb[i] = __float2bfloat16_rn(h);
}

// s[r] = H2[r] . w3 + b3
__global__ void k_output(int rows, const float* __restrict__ H2, const float* __restrict__ w3,
                         const float* __restrict__ b3, float* __restrict__ s) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float acc = 0.f;
  for (int c = 0; c < 128; ++c) acc += H2[static_cast<size_t>(r) * 128 + c] * w3[c];
  s[r] = acc + b3[0];
}

// Listwise softmax cross-entropy per group of rows (a search node's
// candidates): ds = softmax(s) - target; *loss += -sum target * log softmax.
__global__ void k_group_softmax(int n_groups, const int* __restrict__ off,
                                const float* __restrict__ s, const float* __restrict__ target,
                                float* __restrict__ ds, float* __restrict__ loss, float scale) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= n_groups) return;
  const int a = off[gi], b = off[gi + 1];
  float mx = -3.4e38f;
  for (int r = a; r < b; ++r) mx = fmaxf(mx, s[r]);
  float z = 0.f;
  for (int r = a; r < b; ++r) z += __expf(s[r] - mx);
  const float lz = __logf(z) + mx;
  float l = 0.f;
  for (int r = a; r < b; ++r) {
    const float p = __expf(s[r] - lz);
    ds[r] = (p - target[r]) * scale;  // gradient of the mean over groups
    l -= target[r] * (s[r] - lz);
  }
  atomicAdd(loss, l);
}

// dZ2 = ds (x) w3, masked by relu'(layer 2); FP32 and BF16 copies.
__global__ void k_back_out(int rows, const float* __restrict__ ds, const float* __restrict__ w3,
                           const float* __restrict__ H2, float* __restrict__ dZ,
                           __nv_bfloat16* __restrict__ dZb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * 128) return;
  const float v = H2[i] > 0.f ? ds[i >> 7] * w3[i & 127] : 0.f;
  dZ[i] = v;
  dZb[i] = __float2bfloat16_rn(v);
}

// dZ1 = G masked by relu'(layer 1); FP32 and BF16 copies.
__global__ void k_back_relu(int rows, const float* __restrict__ G, const float* __restrict__ H1,
                            float* __restrict__ dZ, __nv_bfloat16* __restrict__ dZb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * 128) return;
  const float v = H1[i] > 0.f ? G[i] : 0.f;
  dZ[i] = v;
  dZb[i] = __float2bfloat16_rn(v);
}

// out[c] = sum_r M[r][c] * (scale ? scale[r] : 1); one block per column.
__global__ void k_colsum(int rows, int cols, const float* __restrict__ M,
                         const float* __restrict__ scale, float* __restrict__ out) {
  const int c = blockIdx.x;
  float acc = 0.f;
  for (int r = threadIdx.x; r < rows; r += blockDim.x)
    acc += M[static_cast<size_t>(r) * cols + c] * (scale ? scale[r] : 1.f);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += part[w];
    out[c] = s;
  }
}

// Adam on the flat parameter vector (inputs 12..15 of W1 stay zero).
__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i < kOffB1 && (i & 15) >= kPolicyFeatures) {
    p[i] = 0.f;
    return;
  }
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// FP32 masters -> BF16 training copies of W1 [128][16], W2 [128][128] and the
// fragment image the search kernels read.
__global__ void k_build_policy(const float* __restrict__ p, __nv_bfloat16* __restrict__ w1b,
                               __nv_bfloat16* __restrict__ w2b, PolicyDev* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 128 * 16) w1b[i] = __float2bfloat16_rn(p[kOffW1 + i]);
  if (i < 128 * 128) w2b[i] = __float2bfloat16_rn(p[kOffW2 + i]);
  if (i < 16 * 32) {  // layer-1 fragments: tile j, lane l
    const int j = i >> 5, l = i & 31, g = l >> 2, t = l & 3, o = 8 * j + g;
    const float* w = p + kOffW1 + 16 * o;
    d->w1[j][l] = make_uint2(pack_bf16x2(w[2 * t], w[2 * t + 1]),
                             pack_bf16x2(w[2 * t + 8], w[2 * t + 9]));
  }
  if (i < 8 * 16 * 32) {  // layer-2 fragments: k-step kk, tile j, lane l
    const int kk = i >> 9, j = (i >> 5) & 15, l = i & 31, g = l >> 2, t = l & 3, o = 8 * j + g;
    const float* w = p + kOffW2 + 128 * o + 16 * kk;
    d->w2[kk][j][l] = make_uint2(pack_bf16x2(w[2 * t], w[2 * t + 1]),
                                 pack_bf16x2(w[2 * t + 8], w[2 * t + 9]));
  }
  if (i < 128) {
    d->b1[i] = p[kOffB1 + i];
    d->b2[i] = p[kOffB2 + i];
    d->w3[i] = p[kOffW3 + i];
  }
  if (i == 0) d->b3 = p[kOffB3];
}

// Features of every branch variable of every store (the search kernels'
// write_features, rounded to BF16 as the network sees them); out is
// [n_stores][n_branch][12].  Stores are joined with the root first.
__global__ void k_policy_features(const uint8_t* __restrict__ image, const int2* __restrict__ root,
                                  int n_stores, int n_vars, const int32_t* __restrict__ lb,
                                  const int32_t* __restrict__ ub, const int32_t* __restrict__ depth,
                                  float* __restrict__ out) {
  const Tab tb = make_tab(image);
  const BranchStatic* bs = reinterpret_cast<const BranchStatic*>(tb.bstat);
  const int nb = tb.n_branch;
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(n_stores) * nb) return;
  const int s = static_cast<int>(i / nb), k = static_cast<int>(i - static_cast<long long>(s) * nb);
  // stores are in the caller's variable order; the table and root in the
  // library's (user_of: the caller's index of each variable, after the root)
  const int32_t* user_of = reinterpret_cast<const int32_t*>(root + n_vars) + n_vars;
  const int v = tb.branch[k];
  const int32_t* l = lb + static_cast<size_t>(s) * n_vars;
  const int32_t* u = ub + static_cast<size_t>(s) * n_vars;
  const int2 R = root[v];
  const int vu = user_of[v];
  const int2 D = make_int2(max(l[vu], R.x), min(u[vu], R.y));
  float prog = 0.f;
  if (tb.objective >= 0) {
    const int2 RO = root[tb.objective];
    prog = static_cast<float>(max(l[user_of[tb.objective]], RO.x) - RO.x) /
           (static_cast<float>(RO.y - RO.x) + 1.f);
  }
  uint32_t row[8];
  write_features(row, k, D, R, bs[k], nb, depth ? depth[s] : 0, prog);
  float* o = out + static_cast<size_t>(i) * kPolicyFeatures;
  for (int c = 0; c < kPolicyFeatures; ++c) {
    const uint32_t w = row[c >> 1];
    const uint16_t h = static_cast<uint16_t>((c & 1) ? (w >> 16) : (w & 0xffffu));
    o[c] = __bfloat162float(__ushort_as_bfloat16(h));
  }
}

// Scores of n feature rows (FP32 [n][12]) by the search kernels' network:
// 16-row chunks per warp, rows staged as BF16 in shared memory.
__global__ void k_policy_score(const PolicyDev* __restrict__ pol, int n,
                               const float* __restrict__ f, float* __restrict__ s) {
  __shared__ uint32_t X[8][16 * 8];  // 8 warps x 16 rows x 8 words
  __shared__ float part[8][256];     // tile parts (mlp_score_tiles)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + warp;
  uint32_t* Xw = X[warp];
  for (int i = lane; i < 16 * 8; i += 32) {
    const int r = 16 * c + (i >> 3), w = i & 7;
    float lo = 0.f, hi = 0.f;
    if (r < n && 2 * w < kPolicyFeatures) lo = f[static_cast<size_t>(r) * kPolicyFeatures + 2 * w];
    if (r < n && 2 * w + 1 < kPolicyFeatures)
      hi = f[static_cast<size_t>(r) * kPolicyFeatures + 2 * w + 1];
    Xw[i] = pack_bf16x2(lo, hi);
  }
  __syncwarp();
  if (16 * c >= n) return;
  mlp_score_tiles(pol, Xw, 0, 0, 16, part[warp]);
  __syncwarp();
  if (lane < 16 && 16 * c + lane < n) s[16 * c + lane] = mlp_row_score(pol, part[warp], lane);
}

}  // namespace pccp
