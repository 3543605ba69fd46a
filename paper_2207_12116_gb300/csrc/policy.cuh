// policy.cuh -- learned branching: per-variable features and a small MLP
// (12 -> 128 -> 128 -> 1, ReLU) that scores the unfixed branch variables of a
// search node.  BF16 weights and activations, FP32 accumulation, on the
// tensor cores through warp-level mma.sync m16n8k16 tiles: the contraction is
// a handful of 16 x 128 x 128 tiles per node inside one team of a persistent
// search kernel, so it is issued by the team's own warps from registers (a
// per-CTA TMEM allocation and single-thread tcgen05 issue would serialise the
// teams that share a CTA for work worth ~1% of a node).
//
// The policy only chooses which variable to split; the split itself (lower
// half first) and the tree it spans are those of the plain strategies, so a
// complete search keeps exact optima whatever the scores are.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "pccp_device.cuh"

namespace pccp {

constexpr int kPolicyFeatures = 12;
constexpr int kPolicyHidden = 128;

// Device image of a policy (built by pccp_policy_create).  B operands are
// stored as ready-made m16n8k16 fragments: two 32-bit words per lane.
struct PolicyDev {
  uint2 w1[16][32];      // layer 1, n-tile j (outputs 8j..8j+7), lane; K = 16 (12 used)
  uint2 w2[8][16][32];   // layer 2, k-step kk (inputs 16kk..), n-tile j, lane
  float b1[kPolicyHidden];
  float b2[kPolicyHidden];
  float w3[kPolicyHidden];
  float b3;
  float pad[3];
};

// Static features of the branch variables (per model, in the table image):
// out-degree and summed offsets of temporal rows (x), in-degree (y), reified
// rows touching the variable, and its demand: the mean, over the reified
// rows b <=> (v <= y < v + d), of the sum of coef / bound over the linear
// rows holding b (for a task's start time: its total demand, the sum over
// resources of usage / capacity).
struct BranchStatic {
  float out_deg, sum_d, in_deg, n_reified, demand, pad[3];
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// The 12 features of branch variable number k (index into the branch list)
// at a node, written as 16 bf16 (4 zero pads) into `row` (8 words).
//   0 (lb - lb0) / (w0 + 1)     1 (ub - lb0) / (w0 + 1)    2 (ub - lb) / (w0 + 1)
//   3 log2(1 + ub - lb) / 16    4 out-degree / 8           5 summed offsets / (w0 + 1)
//   6 in-degree / 8             7 reified rows / 64         8 demand / 4
//   9 k / n_branch              10 depth / (depth + 32)    11 objective progress
// (w0 = root width of the variable; objective progress = (lb(obj) - lb0(obj))
// / (root width of obj + 1), 0 without an objective.)
__device__ __forceinline__ void write_features(uint32_t* row, int k, int2 D, int2 R,
                                               const BranchStatic& s, int n_branch, int depth,
                                               float obj_prog) {
  const float inv = 1.0f / (static_cast<float>(R.y - R.x) + 1.0f);
  const float f0 = static_cast<float>(D.x - R.x) * inv;
  const float f1 = static_cast<float>(D.y - R.x) * inv;
  const float f2 = static_cast<float>(D.y - D.x) * inv;
  const float f3 = __log2f(1.0f + static_cast<float>(D.y - D.x)) * (1.0f / 16.0f);
  const float f4 = s.out_deg * 0.125f;
  const float f5 = s.sum_d * inv;
  const float f6 = s.in_deg * 0.125f;
  const float f7 = s.n_reified * (1.0f / 64.0f);
  const float f8 = s.demand * 0.25f;
  const float f9 = static_cast<float>(k) / static_cast<float>(n_branch);
  const float f10 = static_cast<float>(depth) / (static_cast<float>(depth) + 32.0f);
  row[0] = pack_bf16x2(f0, f1);
  row[1] = pack_bf16x2(f2, f3);
  row[2] = pack_bf16x2(f4, f5);
  row[3] = pack_bf16x2(f6, f7);
  row[4] = pack_bf16x2(f8, f9);
  row[5] = pack_bf16x2(f10, obj_prog);
  row[6] = 0u;
  row[7] = 0u;
}

// Layer 1 of rows 16c .. 16c+15 of X, then the output tiles j0 .. j1-1 of
// layer 2 (8 hidden units each) folded into the output weights: for every
// row and tile, part[16 j + row] = sum over the tile's 8 units of
// relu(h2 + b2) * w3 (two units per lane, then the 4 lanes of a row).  One
// warp; the rows' scores are the tiles' parts summed in tile order
// (mlp_row_score), so the result does not depend on how many warps shared
// the tiles.  Kept out of line so its 40-odd live registers do not raise
// the register count of the propagation loop.
__device__ __noinline__ void mlp_score_tiles(const PolicyDev* __restrict__ pol,
                                             const uint32_t* X, int c, int j0, int j1,
                                             float* part) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = 16 * c + g, r1 = r0 + 8;
  const uint32_t a1[4] = {X[8 * r0 + t], X[8 * r1 + t], X[8 * r0 + 4 + t], X[8 * r1 + 4 + t]};
  uint32_t a2[8][4];
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
    mma_16816(d0, a1, __ldg(&pol->w1[2 * kk][lane]));
    mma_16816(d1, a1, __ldg(&pol->w1[2 * kk + 1][lane]));
    const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
    const float b00 = __ldg(&pol->b1[c0]), b01 = __ldg(&pol->b1[c0 + 1]);
    const float b10 = __ldg(&pol->b1[c1]), b11 = __ldg(&pol->b1[c1 + 1]);
    a2[kk][0] = pack_bf16x2(fmaxf(d0[0] + b00, 0.f), fmaxf(d0[1] + b01, 0.f));
    a2[kk][1] = pack_bf16x2(fmaxf(d0[2] + b00, 0.f), fmaxf(d0[3] + b01, 0.f));
    a2[kk][2] = pack_bf16x2(fmaxf(d1[0] + b10, 0.f), fmaxf(d1[1] + b11, 0.f));
    a2[kk][3] = pack_bf16x2(fmaxf(d1[2] + b10, 0.f), fmaxf(d1[3] + b11, 0.f));
  }
#pragma unroll 1
  for (int j = j0; j < j1; ++j) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) mma_16816(acc, a2[kk], __ldg(&pol->w2[kk][j][lane]));
    const int c0 = 8 * j + 2 * t;
    const float bb0 = __ldg(&pol->b2[c0]), bb1 = __ldg(&pol->b2[c0 + 1]);
    const float w0 = __ldg(&pol->w3[c0]), w1 = __ldg(&pol->w3[c0 + 1]);
    float p_lo = fmaxf(acc[0] + bb0, 0.f) * w0 + fmaxf(acc[1] + bb1, 0.f) * w1;
    float p_hi = fmaxf(acc[2] + bb0, 0.f) * w0 + fmaxf(acc[3] + bb1, 0.f) * w1;
    p_lo += __shfl_xor_sync(0xffffffffu, p_lo, 1);
    p_lo += __shfl_xor_sync(0xffffffffu, p_lo, 2);
    p_hi += __shfl_xor_sync(0xffffffffu, p_hi, 1);
    p_hi += __shfl_xor_sync(0xffffffffu, p_hi, 2);
    if (t == 0) {
      part[16 * j + g] = p_lo;
      part[16 * j + g + 8] = p_hi;
    }
  }
}

// Score of row `row` (0..15) of a chunk from its 16 tile parts, in tile order.
__device__ __forceinline__ float mlp_row_score(const PolicyDev* __restrict__ pol,
                                               const float* part, int row) {
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) s += part[16 * j + row];
  return s + __ldg(&pol->b3);
}

// Order-preserving map of a float score to an unsigned integer.
__device__ __forceinline__ uint32_t score_key(float s) {
  const uint32_t u = __float_as_uint(s);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Selection key of the learned strategy: highest score first, ties to the
// lower branch index; 0 means "no unfixed branch variable".
__device__ __forceinline__ unsigned long long learned_key(float s, int k) {
  return (static_cast<unsigned long long>(score_key(s)) << 32) |
         static_cast<unsigned long long>(0xffffffffu - static_cast<uint32_t>(k));
}

// Learned selection by a whole team after a fixed point: features of every
// branch variable into X (shared memory, 8 words per row, rows padded to a
// multiple of 16; then 256 floats of tile parts per 16-row chunk), a team
// barrier, the warps compute the tile parts of the chunks, a team barrier,
// and the threads sum the parts of the unfixed candidates and submit their
// keys to *sel in the minimum form of the plain strategies (~learned_key:
// its low 32 bits are the branch index).  Words of X per team:
// policy_x_words = 24 * (branch variables rounded up to 16).
__device__ __forceinline__ void learned_select(const Tab& tb, int2* st,
                                               const int2* __restrict__ root, const Team& tm,
                                               const PolicyDev* __restrict__ pol, uint32_t* X,
                                               unsigned long long* sel, int depth) {
  const int nb = tb.n_branch, nbp = (nb + 15) & ~15;
  const BranchStatic* bs = reinterpret_cast<const BranchStatic*>(tb.bstat);
  float prog = 0.f;
  if (tb.objective >= 0) {
    const int2 RO = __ldg(root + tb.objective);
    prog = static_cast<float>(ld_dom(st, tb.objective).x - RO.x) /
           (static_cast<float>(RO.y - RO.x) + 1.f);
  }
  int n_open = 0, last = -1;  // unfixed candidates of this thread
  for (int k = tm.tid; k < nbp; k += tm.nthr) {
    if (k < nb) {
      const int v = tb.branch[k];
      const int2 D = ld_dom(st, v);
      if (D.x < D.y) {
        ++n_open;
        last = k;
      }
      write_features(X + 8 * k, k, D, __ldg(root + v), bs[k], nb, depth, prog);
    } else {
      for (int w = 0; w < 8; ++w) X[8 * k + w] = 0u;
    }
  }
  // with at most one unfixed candidate there is nothing to rank: the network
  // is not run (the choice is the same), which is common near the leaves
  const int holders = team_bar_popc(tm.bar, tm.nthr, n_open > 0);
  if (holders <= 1 && !team_bar_or(tm.bar, tm.nthr, n_open > 1)) {
    if (n_open == 1) atomicMin(sel, static_cast<unsigned long long>(last));
    return;
  }
  // the 16 output tiles of every 16-row chunk, split across the team's warps
  // (S warps per chunk when there are enough); parts after the features in X
  const int n_chunks = nbp / 16;
  int S = 1;
  while (S < 16 && n_chunks * S * 2 <= tm.nwarps) S *= 2;
  float* P = reinterpret_cast<float*>(X + 8 * nbp);  // [n_chunks][16 tiles][16 rows]
  for (int u = tm.warp; u < n_chunks * S; u += tm.nwarps) {
    const int c = u / S, sp = u % S;
    mlp_score_tiles(pol, X, c, sp * (16 / S), (sp + 1) * (16 / S), P + 256 * c);
  }
  team_bar(tm.bar, tm.nthr);
  for (int k = tm.tid; k < nb; k += tm.nthr) {
    const int2 D = ld_dom(st, tb.branch[k]);
    if (D.x < D.y) atomicMin(sel, ~learned_key(mlp_row_score(pol, P + 256 * (k >> 4), k & 15), k));
  }
}

}  // namespace pccp
