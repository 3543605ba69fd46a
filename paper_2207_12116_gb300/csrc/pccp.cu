// pccp.cu -- kernels and C ABI of the PCCP propagate-and-search library (sm_103a).
//
// Kernels
//   k_propagate   : persistent CTAs; the packed propagator table is brought
//                   into shared memory once per CTA by TMA bulk copies; each
//                   team of warps pulls stores from a global counter, stages
//                   one store (joined with the root domains) into shared
//                   memory and runs the lock-free fixed-point loop on it.
//   k_solve       : one team per CTA walks one model's search tree depth first
//                   in the sequential order (Sec. 5: propagate, branch, full
//                   recomputation from the root store on backtrack); CTAs pull
//                   models from a global counter, so a batch of uneven models
//                   balances itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/pccp.h"
#include "pccp_device.cuh"
#include "k_propagate.cuh"
#include "k_solve_eps.cuh"
#include "policy_train.cuh"

using namespace pccp;

namespace {

constexpr int kDefaultMaxIter = 1 << 24;
constexpr int kMaxTeamsPerCta = 15;  // named barriers 1..15
constexpr int32_t kValueLimit = (1 << 30) - 1;
// shared memory a store needs beside its interval slots (control, change
// words): an interval store within this of the limit keeps Booleans as bits
constexpr int64_t kBitStoreSlack = 8192;

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------------ search

struct InstanceDesc {
  const uint8_t* image;
  const int2* root;
  uint32_t image_bytes;
  int32_t n_vars;
  int32_t witness_off;
  int32_t n_branch;
  int32_t max_iter;
  int32_t index;  // the model's position in the caller's list (its result slot)
};

struct InstanceResult {
  int32_t status, has_solution, objective, max_depth;
  int64_t nodes, fails, solutions, iterations;
  int64_t evals;
  int32_t error;
  int32_t us;  // device time of this model's search, microseconds
};

static_assert(sizeof(InstanceDesc) == 40, "descriptor size is part of the scratch accounting");
static_assert(sizeof(InstanceResult) == 64, "result size is part of the scratch accounting");

struct SolveArgs {
  const InstanceDesc* inst;
  InstanceResult* res;
  int32_t* witness;
  int2* stacks;  // [gridDim.x][max_depth]
  int* counter;
  int n_inst;
  int max_depth;
  int mode;
  int strategy;
  int obj_ub;
  int64_t node_limit;
  int64_t time_limit_ns;
  uint32_t max_image_bytes;  // 0 when the tables are read from global memory
  int max_track_words;
  int table_global;
  int stream_stages;          // table_global: buffers of the stream (0: rows read in place)
  int x_words;                // learned strategy: feature rows per team (words)
  int max_vars_smem;          // store slots reserved per CTA
  const PolicyDev* policy;
  // k_solve_slots: teams per CTA, each in a slot of slot_bytes of shared
  // memory: [mbarrier | SearchCtrl | change words | feature rows |
  //          decision stack (max_depth entries) | store | image]
  int team_size;
  int teams;
  uint32_t slot_bytes;
  uint32_t off_track, off_x, off_stack, off_store;  // byte offsets inside a slot
  int levels;  // temporal levels: bit 0 with tables in shared memory, bit 1 in global memory
};

// Broadcast slots of one team's search.  Each slot has one writer (thread 0)
// and one write point per node; it is read right after the barrier that
// follows the write and is not rewritten before another barrier has passed.
struct SearchCtrl {
  unsigned long long sel[2];  // selection key, one slot per node parity
  FixCtrl fc;  // fixed-point failure flag and work counters (reset in P1)
  int stop;    // P1: limit reached
  int record;  // solution path: copy the witness
  int err;     // branch path: decision stack overflow
  int depth;   // backtrack: new depth, -1 when the tree is exhausted
  int next;    // next model index (CTA loop)
  int cur_depth;  // P1: depth of the node (features of the learned strategy)
  int pad;
  // thread 0's search state (shared memory, so that the other threads do
  // not hold it in registers through the fixed point)
  struct {
    int64_t nodes, fails, sols, iters, evals;
    uint64_t t0;
    int depth, max_d, best, objective, error;
    int has_sol, limited, satisfied;
  } ds;
};

constexpr unsigned long long kNoVar = ~0ull;
constexpr uint32_t kRightBit = 0x80000000u;

// Depth-first branch and bound of one model by one team.  Kept out of line:
// k_solve_slots holds two instantiations (staged and in-place tables), and
// separate register allocation for each measured 5% faster on 256 30-60-task
// models (the per-node loop inlined into the queue kernel measured faster
// there, so q_search_item stays inline).
// Each node's store is fix(root join decisions join objective bound); the
// walk order is the sequential one: left child (ub <= m) subtree first.
// All control decisions are made by thread 0 and broadcast through shared
// memory; every broadcast slot is written before a barrier and read after it,
// and never rewritten before the next barrier that follows all its reads.
template <bool kTrack, bool kLearned, bool kGlobal, bool kStream, int kBitSel = kBitsAny>
__device__ __noinline__ void team_dfs(const Tab& tb, const int2* __restrict__ root, int2* st, const Team& tm,
                         SearchCtrl* sc, const Track& tk, int2* stack, const SolveArgs& a,
                         int max_iter, int32_t* witness, InstanceResult* out, uint32_t* X,
                         Streamer* stream) {
  const int nv = tb.n_vars;
  // the root in the store layout (after the root box and the two index maps)
  const int2* root_store = root + 2 * static_cast<size_t>(nv);
  // thread 0's state (only thread 0 reads or writes it)
  auto& S = sc->ds;
  if (tm.tid == 0) {
    S.t0 = globaltimer_ns();
    S.nodes = S.fails = S.sols = S.iters = S.evals = 0;
    S.depth = S.max_d = S.best = S.objective = S.error = 0;
    S.has_sol = S.limited = S.satisfied = 0;
  }
  unsigned par = 0;
  // team-uniform: the store is a fixed point strengthened by marked tells
  // (left descent) rather than a store built from the root
  bool seeded = false;

  for (int v = tm.tid; v < tb.n_slots; v += tm.nthr) st[v] = __ldg(root_store + v);
  if (kTrack) track_clear02(tk, tm);

  for (;;) {
    // P1: limits, objective bound, reset of per-node slots
    if (tm.tid == 0) {
      int stop = 0;
      if (a.node_limit > 0 && S.nodes >= a.node_limit) stop = 1;
      if (a.time_limit_ns > 0 && static_cast<int64_t>(globaltimer_ns() - S.t0) > a.time_limit_ns)
        stop = 1;
      if (!stop && tb.objective >= 0) {
        int bound = a.obj_ub;
        if (a.mode == PCCP_OPTIMISE && S.has_sol) bound = min(bound, S.best - 1);
        if (bound < INT_MAX) {
          const int old = atom_min_s32(&st[tb.objective].y, bound);
          if (kTrack && old > bound) mark_changed(tb, tk, 2, tb.objective);
        }
      }
      S.limited = stop != 0;
      sc->stop = stop;
      sc->fc.fail = 0;
      sc->fc.evals = 0;
      sc->fc.bytes = 0;
      sc->sel[par] = kNoVar;
      sc->cur_depth = S.depth;
    }
    team_bar(tm.bar, tm.nthr);  // N1
    if (sc->stop) break;
    int it = 0;
    const int fst =
        team_fixpoint<kTrack, kGlobal, kStream, kBitSel, true>(tb, st, tm, &sc->fc, tk, !seeded,
                                                         max_iter, it, stream);
    if (tm.tid == 0) {
      ++S.nodes;
      S.iters += it;
      S.evals += sc->fc.evals;
      S.max_d = max(S.max_d, S.depth);
    }
    if (fst == kError) {
      if (tm.tid == 0) {
        S.error = 1;
        S.limited = true;
      }
      break;
    }
    bool backtrack = true;
    if (fst == kFailed) {
      if (tm.tid == 0) ++S.fails;
    } else {
      // A5: variable selection by a team-wide minimum over branch variables
      unsigned long long* sel = &sc->sel[par];
      if (kLearned) {
        learned_select(tb, st, root, tm, a.policy, X, sel, sc->cur_depth);
      } else {
        for (int k = tm.tid; k < tb.n_branch; k += tm.nthr) {
          const int v = tb.branch[k];
          const int2 D = ld_dom(st, v);
          if (D.x < D.y) {
            unsigned long long key = static_cast<unsigned long long>(k);
            if (a.strategy == PCCP_FIRST_FAIL)
              key |= static_cast<unsigned long long>(static_cast<uint32_t>(D.y - D.x)) << 32;
            atomicMin(sel, key);
            if (a.strategy == PCCP_INPUT_ORDER) break;
          }
        }
      }
      if (kTrack) track_clear02(tk, tm);  // for a left child's seeded fixed point
      team_bar(tm.bar, tm.nthr);  // N2
      const unsigned long long key = *sel;
      if (key == kNoVar) {  // every branch variable fixed: a solution
        if (tm.tid == 0) {
          ++S.sols;
          const int z = tb.objective >= 0 ? st[tb.objective].x : 0;
          const bool record = (a.mode == PCCP_OPTIMISE) || !S.has_sol;
          if (record) {
            S.best = z;
            S.objective = z;
          }
          S.has_sol = true;
          if (a.mode == PCCP_OPTIMISE && tb.objective < 0) S.satisfied = true;
          sc->record = record;
        }
        team_bar(tm.bar, tm.nthr);  // N3
        if (sc->record) {  // in the caller's variable order (internal_of after the root)
          const int32_t* internal_of = reinterpret_cast<const int32_t*>(root + nv);
          for (int x = tm.tid; x < nv; x += tm.nthr)
            witness[x] = var_dom_plain(st, tb.bit0, __ldg(internal_of + x)).x;
        }
      } else {
        backtrack = false;
        if (tm.tid == 0) {
          const int v = tb.branch[static_cast<int>(key & 0xffffffffull)];
          const int2 D = st[v];
          const int m = D.x + (D.y - D.x) / 2;
          if (S.depth >= a.max_depth) {
            S.error = 2;
          } else {
            stack[S.depth] = make_int2(v, m);  // left: ub(v) <= m
            ++S.depth;
            atom_min_s32(&st[v].y, m);  // m < ub(v): always a change
            if (kTrack) mark_changed(tb, tk, 2, v);
          }
          sc->err = S.error != 0;
        }
        team_bar(tm.bar, tm.nthr);  // NB: publishes the error decision
        if (sc->err) {
          if (tm.tid == 0) S.limited = true;
          break;
        }
        seeded = true;
      }
    }
    par ^= 1u;
    if (backtrack) {
      if (tm.tid == 0) {
        while (S.depth > 0 && (static_cast<uint32_t>(stack[S.depth - 1].x) & kRightBit)) --S.depth;
        if (S.depth == 0 || S.satisfied) {
          sc->depth = -1;
        } else {
          const int2 e = stack[S.depth - 1];  // flip to the right child: lb(v) >= m + 1
          stack[S.depth - 1] = make_int2(static_cast<int>(static_cast<uint32_t>(e.x) | kRightBit),
                                       e.y + 1);
          sc->depth = S.depth;
        }
      }
      team_bar(tm.bar, tm.nthr);  // N4
      const int d = sc->depth;
      if (d < 0) break;
      for (int v = tm.tid; v < tb.n_slots; v += tm.nthr) st[v] = __ldg(root_store + v);
      if (kTrack) track_clear02(tk, tm);
      seeded = false;
      team_bar(tm.bar, tm.nthr);  // N5
      for (int k = tm.tid; k < d; k += tm.nthr) {
        const int2 e = stack[k];
        const int v = static_cast<int>(static_cast<uint32_t>(e.x) & ~kRightBit);
        if (static_cast<uint32_t>(e.x) & kRightBit)
          atom_max_s32(&st[v].x, e.y);
        else
          atom_min_s32(&st[v].y, e.y);
      }
    }
  }
  if (tm.tid == 0) {
    out->status = S.limited ? PCCP_RES_LIMIT : (S.has_sol ? PCCP_RES_OPTIMAL : PCCP_RES_INFEASIBLE);
    out->has_solution = S.has_sol;
    out->objective = S.has_sol ? S.objective : 0;
    out->max_depth = S.max_d;
    out->nodes = S.nodes;
    out->fails = S.fails;
    out->solutions = S.sols;
    out->iterations = S.iters;
    out->evals = S.evals;
    out->error = S.error;
    {
      const uint64_t us = (globaltimer_ns() - S.t0) / 1000u;
      out->us = us > 0x7fffffffull ? 0x7fffffff : static_cast<int32_t>(us);
    }
  }
}

template <bool kTrack, bool kLearned, bool kGlobal, bool kStream>
__global__ void __launch_bounds__(1024) k_solve(SolveArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  // [table image | kGlobal: the stream region, or none][mbarrier][SearchCtrl]
  // [change words][store][feature rows]
  const size_t head = kGlobal ? stream_bytes(a.stream_stages) : a.max_image_bytes;

  uint8_t* img = smem;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + head);
  SearchCtrl* sc = reinterpret_cast<SearchCtrl*>(smem + head + 16);
  uint32_t* track_base =
      reinterpret_cast<uint32_t*>(smem + head + 16 + sizeof(SearchCtrl));
  int2* st = reinterpret_cast<int2*>(track_base + ((a.max_track_words + 3) & ~3));
  uint32_t* X = reinterpret_cast<uint32_t*>(st + a.max_vars_smem);
  if (threadIdx.x == 0) mbar_init(mbar, 1);
  Team tm;
  tm.tid = threadIdx.x;
  tm.nthr = blockDim.x;
  tm.bar = 1;
  tm.lane = threadIdx.x & 31;
  tm.warp = threadIdx.x >> 5;
  tm.nwarps = blockDim.x >> 5;
  int2* stack = a.stacks + static_cast<size_t>(blockIdx.x) * a.max_depth;
  uint32_t parity = 0;
  Streamer stream;
  bool open = false;
  uint32_t seq = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) sc->next = atomicAdd(a.counter, 1);
    __syncthreads();
    const int i = sc->next;
    if (i >= a.n_inst) break;
    const InstanceDesc d = a.inst[i];
    if (!kGlobal) {
      if (!load_image(img, d.image, d.image_bytes, mbar, parity)) {
        if (threadIdx.x == 0) {
          a.res[d.index].status = PCCP_RES_LIMIT;
          a.res[d.index].error = 3;
        }
        return;
      }
      parity ^= 1u;
    } else {
      __syncthreads();
    }
    const Tab tb = make_tab(kGlobal ? d.image : img, a.levels & (kGlobal ? 2 : 1));
    const Track tk = make_track(track_base, tb.n_vars, tb.n_lin + tb.n_lin_long);
    if (kStream) {  // the previous model's prefetched copies land first
      if (open) seq = stream_close(stream);
      stream = stream_open(img, a.stream_stages, tb, d.image, tm, seq);
      open = true;
      __syncthreads();
    }
    team_dfs<kTrack, kLearned, kGlobal, kStream>(tb, d.root, st, tm, sc, tk, stack, a,
                                                 d.max_iter, a.witness + d.witness_off,
                                                 &a.res[d.index], X, &stream);
  }
  if (kStream && open) stream_close(stream);
}

// Copy a table image prefix into a team's shared memory by TMA bulk copies
// issued by the team's thread 0; every thread of the team waits (bounded) for
// completion on the team's mbarrier.  The team barrier at the start orders
// the team's earlier generic reads of dst before the async-proxy writes.
// Returns the same value on every thread of the team: false if the wait gave
// up (the caller must then not read dst).
__device__ __forceinline__ bool team_load_image(uint8_t* dst, const uint8_t* src, uint32_t bytes,
                                                uint64_t* mbar, uint32_t parity, const Team& tm) {
  team_bar(tm.bar, tm.nthr);
  if (tm.tid == 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(mbar, bytes);
    const uint32_t chunk = 32768;
    for (uint32_t o = 0; o < bytes; o += chunk) {
      const uint32_t n = (bytes - o < chunk) ? (bytes - o) : chunk;
      bulk_copy_g2s(dst + o, src + o, n, mbar);
    }
  }
  bool ok = mbar_wait_bounded(mbar, parity, 1 << 22);
  if (!ok) ok = mbar_wait_bounded(mbar, parity, 1 << 22);  // drain before giving up
  return !team_bar_or(tm.bar, tm.nthr, !ok);
}

// Batched depth-first search with several teams per CTA (a.teams slots of
// a.team_size threads).  Each team pulls models from the global queue (the
// host orders it largest table first) and searches each one alone in the
// sequential order (team_dfs), so every model's node counts are those of
// the one-team search.  A model whose table prefix fits in the slot beside
// its store is staged there by TMA bulk copies; a larger one is read in
// place from the device image (through L1 / L2), which is where its change
// tracking pays (kTrackS / kTrackG: skip stable rows for tables in shared /
// global memory).
template <bool kTrackS, bool kTrackG, bool kLearned>
__global__ void __launch_bounds__(1024) k_solve_slots(SolveArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int team_id = threadIdx.x / a.team_size;
  uint8_t* slot = smem + static_cast<size_t>(team_id) * a.slot_bytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(slot);
  SearchCtrl* sc = reinterpret_cast<SearchCtrl*>(slot + 16);
  uint32_t* track_base = reinterpret_cast<uint32_t*>(slot + a.off_track);
  uint32_t* X = reinterpret_cast<uint32_t*>(slot + a.off_x);
  int2* st = reinterpret_cast<int2*>(slot + a.off_store);
  Team tm;
  tm.tid = threadIdx.x - team_id * a.team_size;
  tm.nthr = a.team_size;
  tm.bar = 1 + team_id;
  tm.lane = threadIdx.x & 31;
  tm.warp = tm.tid >> 5;
  tm.nwarps = a.team_size >> 5;
  if (tm.tid == 0) {
    mbar_init(mbar, 1);
    fence_mbarrier_init();
  }
  int2* stack = reinterpret_cast<int2*>(slot + a.off_stack);
  uint32_t parity = 0;
  for (;;) {
    team_bar(tm.bar, tm.nthr);  // the previous model is done (first pass: mbarrier ready)
    if (tm.tid == 0) sc->next = atomicAdd(a.counter, 1);
    team_bar(tm.bar, tm.nthr);
    const int q = sc->next;
    if (q >= a.n_inst) break;
    const InstanceDesc d = a.inst[q];
    InstanceResult* out = &a.res[d.index];
    const TableHeader* hg = reinterpret_cast<const TableHeader*>(d.image);
    // the image prefix after the store, 128-byte aligned, when it fits
    const uint32_t img_off =
        (a.off_store + 8u * static_cast<uint32_t>(__ldg(&hg->n_slots)) + 127u) & ~127u;
    const uint32_t copy = static_cast<uint32_t>(kTrackS ? __ldg(&hg->track_bytes)
                                                        : __ldg(&hg->core_bytes));
    // models keeping Booleans as bits are read in place (only the
    // global-table instantiations read that layout)
    if (img_off + copy <= a.slot_bytes && __ldg(&hg->bit0) == d.n_vars) {
      uint8_t* img = slot + img_off;
      if (!team_load_image(img, d.image, copy, mbar, parity, tm)) {
        if (tm.tid == 0) {
          out->status = PCCP_RES_LIMIT;
          out->error = 3;
        }
        return;  // this team stops; its mbarrier phase may still be pending
      }
      parity ^= 1u;
      Tab tb = make_tab(img, a.levels & 1);
      tb.lin_shift = lin_split_shift(tb, tm.nthr);
      const Track tk = make_track(track_base, tb.n_vars, tb.n_lin + tb.n_lin_long);
      team_dfs<kTrackS, kLearned, false, false>(tb, d.root, st, tm, sc, tk, stack, a, d.max_iter,
                                                a.witness + d.witness_off, out, X, nullptr);
    } else {
      Tab tb = make_tab(d.image, a.levels & 2);
      // the temporal levels (a few KB walked as chains of dependent loads)
      // into the slot after the store when they fit, else read in place
      const uint32_t tl_off = static_cast<uint32_t>(__ldg(&hg->off_tlev));
      const uint32_t tl = static_cast<uint32_t>(__ldg(&hg->core_bytes)) - tl_off;
      if (tb.n_tlev > 0 && img_off + tl <= a.slot_bytes) {
        if (!team_load_image(slot + img_off, d.image + tl_off, tl, mbar, parity, tm)) {
          if (tm.tid == 0) {
            out->status = PCCP_RES_LIMIT;
            out->error = 3;
          }
          return;
        }
        parity ^= 1u;
        tab_levels_at(tb, slot + img_off);
      }
      const Track tk = make_track(track_base, tb.n_vars, tb.n_lin + tb.n_lin_long);
      // one compilation each for models with and without Booleans as bits
      if (tb.bit0 < tb.n_vars)
        team_dfs<kTrackG, kLearned, true, false, kBitsYes>(tb, d.root, st, tm, sc, tk, stack, a,
                                                           d.max_iter, a.witness + d.witness_off,
                                                           out, X, nullptr);
      else
        team_dfs<kTrackG, kLearned, true, false, kBitsNo>(tb, d.root, st, tm, sc, tk, stack, a,
                                                          d.max_iter, a.witness + d.witness_off,
                                                          out, X, nullptr);
    }
  }
}

#include "k_search_queue.inc"

// -------------------------------------------------------------- host model

struct Packed {
  std::vector<uint8_t> image;  // header + sections, 16-byte aligned sizes
  int32_t n_vars, n_t, n_rf, n_lin, n_terms, n_branch, objective;
  int32_t n_seg;
  int64_t bytes_per_sweep;
  uint32_t core_bytes, track_bytes;  // image prefixes copied to shared memory
  int32_t bit0, n_slots;             // store layout
  int32_t n_tlev;                    // levels of the temporal rows (0: not acyclic)
  uint32_t tlev_bytes;               // their section (the end of the core prefix)
};

size_t align16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

// Where the temporal levels run (bit 0: tables in shared memory, bit 1:
// tables in global memory) for an option value (1 on, -1 off, 0 the
// library's choice: everywhere in propagation, global tables in searches).
int levels_mask(int32_t opt, bool propagation) {
  return opt > 0 ? 3 : opt < 0 ? 0 : (propagation ? 3 : 2);
}

}  // namespace

struct pccp_policy;
namespace {
int policy_device(const pccp_policy* p);
const PolicyDev* policy_dev(const pccp_policy* p);
}  // namespace

struct HostPipe;

struct pccp_model {
  int device;
  int32_t n_vars, n_t, n_rf, n_lin, n_terms, n_branch, objective;
  int32_t n_seg;  // stream segments of the table
  int32_t reordered;  // 1: shared-memory stores use the library's variable order
  uint32_t image_bytes;  // whole image (read in place from global memory)
  uint32_t core_bytes;   // prefix copied to shared memory by kernels without change tracking
  uint32_t track_bytes;  // prefix copied by kernels that skip stable rows
  int64_t bytes_per_sweep;
  int32_t max_iter;  // every changing iteration narrows some bound by >= 1
  int32_t max_decisions;  // bound on a search path's length (decision stack entries)
  int32_t bit0, n_slots;  // store layout: Booleans from bit0 on as bits; int2 slots per store
  int32_t n_tlev;         // levels of the temporal rows (0: not acyclic)
  uint32_t tlev_bytes;    // their section, the last tlev_bytes of the core prefix
  uint8_t* d_mem;    // image, then root int2[n_vars]
  int2* d_root;
  HostPipe* pipe = nullptr;  // pccp_propagate_host's streams and slots (lazy)
  std::mutex pipe_mu;               // one host-memory propagation at a time
};

namespace {

void host_pipe_free(HostPipe* p);  // pccp_host.inc

int64_t iabs64(int64_t x) { return x < 0 ? -x : x; }

// Reified rows {x | y << 16, b | d << 16} (sorted by b) that pair up: rows
// over the same two variables with the roles swapped, matched first come
// first served; returns (first row, second row) in the order of the first.
std::vector<std::pair<size_t, size_t>> reified_pairs(const std::vector<uint2>& RF) {
  std::vector<std::pair<size_t, size_t>> out;
  std::unordered_map<uint32_t, std::vector<size_t>> waiting;  // (x | y << 16) -> rows
  std::vector<char> used(RF.size(), 0);
  for (size_t r = 0; r < RF.size(); ++r) waiting[RF[r].x].push_back(r);
  for (size_t r = 0; r < RF.size(); ++r) {
    if (used[r]) continue;
    const uint32_t x = RF[r].x & 0xffffu, y = RF[r].x >> 16;
    if (x == y) continue;
    auto it = waiting.find(y | (x << 16));
    if (it == waiting.end()) continue;
    for (size_t q : it->second) {
      if (used[q] || q == r) continue;
      used[r] = used[q] = 1;
      out.emplace_back(r, q);
      break;
    }
  }
  return out;
}

// Shared-memory wavefronts of one warp's 8-byte interval loads of the
// variables vars[0..n) (one per lane, n <= 32) under the order iof: per
// half-warp (128 bytes a wavefront), the largest number of distinct words
// that fall in one of the 32 four-byte banks.
int warp_wavefronts(const int32_t* vars, int n, const std::vector<int32_t>& iof) {
  int total = 0;
  for (int h = 0; h < n; h += 16) {
    uint32_t words[32];
    int nw = 0;
    for (int l = h; l < std::min(n, h + 16); ++l) {
      const uint32_t w = 2u * static_cast<uint32_t>(iof[vars[l]]);
      words[nw++] = w;
      words[nw++] = w + 1;
    }
    std::sort(words, words + nw);
    int per_bank[32] = {0};
    int worst = 0;
    for (int i = 0; i < nw; ++i) {
      if (i > 0 && words[i] == words[i - 1]) continue;  // one word, one access
      worst = std::max(worst, ++per_bank[words[i] % 32]);
    }
    total += worst;
  }
  return total;
}

// Wavefronts of the interval loads of one sweep in the kernels' row order
// (reified pairs and single rows by thread, short linear rows by thread in
// tiles of 32 sorted longest first, long rows by warp; temporal rows are few
// and left out), under the order iof.
int64_t sweep_wavefronts(const pccp_model_desc* d, const std::vector<uint2>& RF,
                         const std::vector<std::pair<size_t, size_t>>& pairs,
                         const std::vector<int32_t>& iof) {
  int64_t total = 0;
  int32_t lanes[4][32];
  for (size_t g = 0; g < pairs.size(); g += 32) {
    const int n = static_cast<int>(std::min<size_t>(32, pairs.size() - g));
    for (int l = 0; l < n; ++l) {
      const uint2 r1 = RF[pairs[g + l].first], r2 = RF[pairs[g + l].second];
      lanes[0][l] = static_cast<int32_t>(r1.x & 0xffffu);
      lanes[1][l] = static_cast<int32_t>(r1.x >> 16);
      lanes[2][l] = static_cast<int32_t>(r1.y & 0xffffu);
      lanes[3][l] = static_cast<int32_t>(r2.y & 0xffffu);
    }
    for (int k = 0; k < 4; ++k) total += warp_wavefronts(lanes[k], n, iof);
  }
  if (d->n_linear <= 0) return total;
  std::vector<std::vector<int32_t>> rows;
  for (int32_t i = 0; i < d->n_linear; ++i) {
    std::vector<int32_t> t;
    for (int32_t k = d->linear_off[i]; k < d->linear_off[i + 1]; ++k)
      if (d->term_coef[k] != 0) t.push_back(d->term_var[k]);
    rows.push_back(std::move(t));
  }
  std::vector<const std::vector<int32_t>*> shorts;
  for (const auto& r : rows) {
    if (r.size() <= static_cast<size_t>(kShortRow)) {
      shorts.push_back(&r);
    } else {
      for (size_t k = 0; k < r.size(); k += 32)
        total += warp_wavefronts(r.data() + k, static_cast<int>(std::min<size_t>(32, r.size() - k)),
                                 iof);
    }
  }
  std::stable_sort(shorts.begin(), shorts.end(),
                   [](const std::vector<int32_t>* p, const std::vector<int32_t>* q) {
                     return p->size() > q->size();
                   });
  for (size_t t0 = 0; t0 < shorts.size(); t0 += 32) {
    const size_t t1 = std::min(shorts.size(), t0 + 32);
    for (size_t k = 0; k < shorts[t0]->size(); ++k) {
      int n = 0;
      for (size_t r = t0; r < t1; ++r)
        if (k < shorts[r]->size()) lanes[0][n++] = (*shorts[r])[k];
      total += warp_wavefronts(lanes[0], n, iof);
    }
  }
  return total;
}

// The library's own numbering of a model's variables (internal_of[user]).
// Stores are kept in shared memory in this order.  Candidates: the caller's
// order, and the pair-block order -- every variable that is the Boolean of no
// reified pair first, in the caller's order, then the first Booleans of the
// pairs in pair order, then the second ones, so that neighbouring lanes that
// evaluate neighbouring pairs load neighbouring words (in the caller's order
// one of the two Booleans may sit a model's width apart, every lane on the
// same banks; a linear row over one column of a matrix of Booleans strides
// by its width too).  The one whose sweep has fewer shared-memory wavefronts
// (sweep_wavefronts) is kept.  The caller's order stays the interface:
// stores are read and written, and witnesses written, through this map.
// Identity when the model has an index out of range (validation reports it).
// Booleans that may be kept as bits (2 bits of a shared 64-bit slot instead
// of an int2 each): variables with a 0/1 root domain that appear only as the
// b of reified rows and as terms of linear rows whose coefficients are all
// positive and whose variables are all 0/1 at the root (the overlap Booleans
// and resource sums of the scheduling model), never as a branch variable,
// the objective, or an operand of another row.  Every reified b and every
// term of such a linear row must then be one of them, else the model keeps
// every variable as an interval (empty result).  Indices are the caller's.
std::vector<char> bit_vars(const pccp_model_desc* d) {
  const int32_t nv = d->n_vars;
  if (nv <= 0 || nv > 65535 || !d->lb0 || !d->ub0) return {};
  if (d->n_temporal < 0 || d->n_reified < 0 || d->n_linear < 0 || d->n_branch < 0) return {};
  if ((d->n_temporal > 0 && !d->temporal) || (d->n_reified > 0 && !d->reified) ||
      (d->n_branch > 0 && !d->branch_vars))
    return {};
  if (d->n_linear > 0 && (!d->linear_c || !d->linear_off || !d->term_var || !d->term_coef ||
                          d->linear_off[0] != 0))
    return {};
  auto ok = [nv](int32_t v) { return v >= 0 && v < nv; };
  std::vector<char> bit(nv, 0);
  for (int32_t v = 0; v < nv; ++v) bit[v] = d->lb0[v] >= 0 && d->ub0[v] <= 1 && d->lb0[v] <= d->ub0[v];
  for (int32_t k = 0; k < d->n_branch; ++k) {
    if (!ok(d->branch_vars[k])) return {};
    bit[d->branch_vars[k]] = 0;
  }
  if (d->objective >= 0) {
    if (!ok(d->objective)) return {};
    bit[d->objective] = 0;
  }
  for (int32_t i = 0; i < d->n_temporal; ++i)
    for (int c = 0; c < 2; ++c) {
      if (!ok(d->temporal[3 * i + c])) return {};
      bit[d->temporal[3 * i + c]] = 0;
    }
  for (int32_t i = 0; i < d->n_reified; ++i)
    for (int c = 0; c < 3; ++c)
      if (!ok(d->reified[4 * i + c])) return {};
  for (int32_t i = 0; i < d->n_reified; ++i)
    for (int c = 1; c < 3; ++c) bit[d->reified[4 * i + c]] = 0;
  std::vector<char> zero_one_row(d->n_linear > 0 ? d->n_linear : 0, 1);
  for (int32_t i = 0; i < d->n_linear; ++i) {
    if (d->linear_off[i + 1] < d->linear_off[i]) return {};
    for (int32_t k = d->linear_off[i]; k < d->linear_off[i + 1]; ++k) {
      const int32_t v = d->term_var[k], a = d->term_coef[k];
      if (!ok(v)) return {};
      if (a == 0) continue;
      if (a < 0 || d->lb0[v] < 0 || d->ub0[v] > 1) zero_one_row[i] = 0;
    }
  }
  for (int32_t i = 0; i < d->n_linear; ++i)
    if (!zero_one_row[i])
      for (int32_t k = d->linear_off[i]; k < d->linear_off[i + 1]; ++k)
        if (d->term_coef[k] != 0) bit[d->term_var[k]] = 0;
  for (int32_t i = 0; i < d->n_reified; ++i)
    if (!bit[d->reified[4 * i]]) return {};
  for (int32_t i = 0; i < d->n_linear; ++i)
    if (zero_one_row[i])
      for (int32_t k = d->linear_off[i]; k < d->linear_off[i + 1]; ++k)
        if (d->term_coef[k] != 0 && !bit[d->term_var[k]]) return {};
  return bit;
}

// Order with Booleans kept as bits: the other variables first (caller's
// order), then the Booleans: the first Booleans of reified pairs in pair
// order, then the second ones, then the rest (neighbouring lanes that
// evaluate neighbouring pairs then read bits of the same slot).
std::vector<int32_t> bit_order(const pccp_model_desc* d, const std::vector<char>& bit) {
  const int32_t nv = d->n_vars;
  std::vector<int32_t> iof(nv);
  std::vector<uint2> RF;
  for (int32_t i = 0; i < d->n_reified; ++i)
    RF.push_back(make_uint2(static_cast<uint32_t>(d->reified[4 * i + 1]) |
                                (static_cast<uint32_t>(d->reified[4 * i + 2]) << 16),
                            static_cast<uint32_t>(d->reified[4 * i])));
  std::stable_sort(RF.begin(), RF.end(),
                   [](const uint2& p, const uint2& q) { return (p.y & 0xffffu) < (q.y & 0xffffu); });
  std::vector<int32_t> rank(nv, 2);  // 0 first Booleans, 1 second ones, 2 the rest
  std::vector<int32_t> first, second;
  for (const auto& pq : reified_pairs(RF)) {
    const int32_t b1 = static_cast<int32_t>(RF[pq.first].y & 0xffffu);
    const int32_t b2 = static_cast<int32_t>(RF[pq.second].y & 0xffffu);
    if (rank[b1] == 2) {
      rank[b1] = 0;
      first.push_back(b1);
    }
    if (rank[b2] == 2) {
      rank[b2] = 1;
      second.push_back(b2);
    }
  }
  int32_t next = 0;
  for (int32_t v = 0; v < nv; ++v)
    if (!bit[v]) iof[v] = next++;
  for (int32_t v : first) iof[v] = next++;
  for (int32_t v : second) iof[v] = next++;
  for (int32_t v = 0; v < nv; ++v)
    if (bit[v] && rank[v] == 2) iof[v] = next++;
  return iof;
}

std::vector<int32_t> internal_order(const pccp_model_desc* d) {
  const int32_t nv = d->n_vars;
  std::vector<int32_t> iof(nv > 0 ? nv : 0);
  for (int32_t v = 0; v < nv; ++v) iof[v] = v;
  if (nv <= 0 || nv > 65535 || d->n_reified <= 0 || !d->reified) return iof;
  if (d->n_linear < 0 || (d->n_linear > 0 && (!d->linear_off || !d->term_var || !d->term_coef)))
    return iof;
  for (int32_t i = 0; i < d->n_linear; ++i)
    if (d->linear_off[0] != 0 || d->linear_off[i + 1] < d->linear_off[i]) return iof;
  for (int32_t k = 0; d->n_linear > 0 && k < d->linear_off[d->n_linear]; ++k)
    if (d->term_var[k] < 0 || d->term_var[k] >= nv) return iof;
  std::vector<uint2> RF;
  for (int32_t i = 0; i < d->n_reified; ++i) {
    const int32_t b = d->reified[4 * i], x = d->reified[4 * i + 1], y = d->reified[4 * i + 2];
    if (b < 0 || b >= nv || x < 0 || x >= nv || y < 0 || y >= nv) return iof;
    RF.push_back(make_uint2(static_cast<uint32_t>(x) | (static_cast<uint32_t>(y) << 16),
                            static_cast<uint32_t>(b)));
  }
  std::stable_sort(RF.begin(), RF.end(),
                   [](const uint2& p, const uint2& q) { return (p.y & 0xffffu) < (q.y & 0xffffu); });
  const auto pairs = reified_pairs(RF);
  if (pairs.empty()) return iof;
  std::vector<int32_t> block(nv, 0);  // 0 rest, 1 first Booleans, 2 second ones
  std::vector<int32_t> first, second;
  for (const auto& pq : pairs) {
    const int32_t b1 = static_cast<int32_t>(RF[pq.first].y & 0xffffu);
    const int32_t b2 = static_cast<int32_t>(RF[pq.second].y & 0xffffu);
    if (block[b1] == 0) {
      block[b1] = 1;
      first.push_back(b1);
    }
    if (block[b2] == 0) {
      block[b2] = 2;
      second.push_back(b2);
    }
  }
  std::vector<int32_t> blocks(nv);
  int32_t next = 0;
  for (int32_t v = 0; v < nv; ++v)
    if (block[v] == 0) blocks[v] = next++;
  for (int32_t v : first) blocks[v] = next++;
  for (int32_t v : second) blocks[v] = next++;
  return sweep_wavefronts(d, RF, pairs, blocks) < sweep_wavefronts(d, RF, pairs, iof) ? blocks
                                                                                       : iof;
}

int validate_and_pack(const pccp_model_desc* d, Packed* p, int32_t bit0 = -1) {
  if (!d) return PCCP_ERR_INVALID;
  const int64_t nv = d->n_vars;
  if (nv < 1) return PCCP_ERR_INVALID;
  if (nv > 65535) return PCCP_ERR_UNSUPPORTED;
  if (!d->lb0 || !d->ub0) return PCCP_ERR_INVALID;
  std::vector<int64_t> B(nv);
  for (int64_t v = 0; v < nv; ++v) {
    if (d->lb0[v] > d->ub0[v]) return PCCP_ERR_INVALID;
    if (d->lb0[v] < -kValueLimit || d->ub0[v] > kValueLimit) return PCCP_ERR_OVERFLOW;
    B[v] = std::max(iabs64(d->lb0[v]), iabs64(d->ub0[v]));
  }
  auto in_range = [nv](int64_t v) { return v >= 0 && v < nv; };
  if (d->n_temporal < 0 || d->n_linear < 0 || d->n_reified < 0 || d->n_branch < 0)
    return PCCP_ERR_INVALID;
  if (d->n_temporal > 0 && !d->temporal) return PCCP_ERR_INVALID;
  if (d->n_reified > 0 && !d->reified) return PCCP_ERR_INVALID;
  if (d->n_linear > 0 && (!d->linear_c || !d->linear_off)) return PCCP_ERR_INVALID;
  if (d->n_branch > 0 && !d->branch_vars) return PCCP_ERR_INVALID;
  if (d->objective < -1 || d->objective >= nv) return PCCP_ERR_INVALID;
  for (int32_t k = 0; k < d->n_branch; ++k)
    if (!in_range(d->branch_vars[k])) return PCCP_ERR_INVALID;

  std::vector<uint2> T, RF;
  struct LinRow {
    int32_t c;
    std::vector<uint32_t> terms;
  };
  std::vector<LinRow> short_rows, long_rows;
  int32_t n_terms = 0;
  int64_t bytes_per_sweep = 0;
  for (int32_t i = 0; i < d->n_temporal; ++i) {
    const int32_t x = d->temporal[3 * i], y = d->temporal[3 * i + 1], dd = d->temporal[3 * i + 2];
    if (!in_range(x) || !in_range(y)) return PCCP_ERR_INVALID;
    if (dd < -kValueLimit || dd > kValueLimit) return PCCP_ERR_OVERFLOW;
    T.push_back(make_uint2(static_cast<uint32_t>(x) | (static_cast<uint32_t>(y) << 16),
                           static_cast<uint32_t>(dd)));
    bytes_per_sweep += 20;
  }
  for (int32_t i = 0; i < d->n_reified; ++i) {
    const int32_t b = d->reified[4 * i], x = d->reified[4 * i + 1], y = d->reified[4 * i + 2],
                  dd = d->reified[4 * i + 3];
    if (!in_range(b) || !in_range(x) || !in_range(y)) return PCCP_ERR_INVALID;
    if (d->lb0[b] < 0 || d->ub0[b] > 1) return PCCP_ERR_INVALID;
    if (dd < -32768 || dd > 32767) return PCCP_ERR_UNSUPPORTED;
    RF.push_back(make_uint2(static_cast<uint32_t>(x) | (static_cast<uint32_t>(y) << 16),
                            static_cast<uint32_t>(b) |
                                (static_cast<uint32_t>(static_cast<uint16_t>(dd)) << 16)));
    bytes_per_sweep += 40;
  }
  // Reified rows sorted by their Boolean: rows evaluated side by side by one
  // warp then touch neighbouring variables (fewer shared-memory bank
  // conflicts).  Row order never changes the fixed point (Sec. 3).
  std::stable_sort(RF.begin(), RF.end(),
                   [](const uint2& p, const uint2& q) { return (p.y & 0xffffu) < (q.y & 0xffffu); });
  // Rows over the same two variables with the roles swapped are evaluated
  // together (one load of x and y for both); the rest stay single.
  std::vector<uint4> RFP;
  {
    std::vector<uint2> single;
    std::vector<char> used(RF.size(), 0);
    for (const auto& pq : reified_pairs(RF)) {
      used[pq.first] = used[pq.second] = 1;
      RFP.push_back(make_uint4(RF[pq.first].x, RF[pq.first].y, RF[pq.second].y, 0u));
    }
    for (size_t r = 0; r < RF.size(); ++r)
      if (!used[r]) single.push_back(RF[r]);
    RF.swap(single);
  }
  if (d->n_linear > 0 && d->linear_off[0] != 0) return PCCP_ERR_INVALID;
  for (int32_t i = 0; i < d->n_linear; ++i) {
    const int32_t o0 = d->linear_off[i], o1 = d->linear_off[i + 1];
    if (o1 < o0) return PCCP_ERR_INVALID;
    if (o1 > o0 && (!d->term_coef || !d->term_var)) return PCCP_ERR_INVALID;
    const int64_t c = d->linear_c[i];
    int64_t sum = 0, mx = 0;
    LinRow row;
    row.c = static_cast<int32_t>(c);
    for (int32_t k = o0; k < o1; ++k) {
      const int32_t a = d->term_coef[k], v = d->term_var[k];
      if (!in_range(v)) return PCCP_ERR_INVALID;
      if (a == 0) continue;
      if (a < -32768 || a > 32767) return PCCP_ERR_UNSUPPORTED;
      sum += iabs64(a) * B[v];
      mx = std::max(mx, iabs64(a) * B[v]);
      row.terms.push_back(static_cast<uint32_t>(v) |
                          (static_cast<uint32_t>(static_cast<uint16_t>(a)) << 16));
    }
    const int32_t len = static_cast<int32_t>(row.terms.size());
    if (len == 0) return PCCP_ERR_INVALID;
    if (iabs64(c) + 2 * sum + 2 * mx > static_cast<int64_t>(INT32_MAX)) return PCCP_ERR_OVERFLOW;
    bytes_per_sweep += 12 + 12 * static_cast<int64_t>(len);
    n_terms += len;
    (len <= kShortRow ? short_rows : long_rows).push_back(std::move(row));
  }
  // Short rows: longest first so each 32-row tile holds rows of similar
  // length; tiles transposed (term t of lane l at tile start + 32 t + l).
  std::stable_sort(short_rows.begin(), short_rows.end(), [](const LinRow& p, const LinRow& q) {
    return p.terms.size() > q.terms.size();
  });
  std::vector<int4> L, LL;
  std::vector<uint32_t> TERMS, TERMS_LONG;
  std::vector<size_t> tile_start;  // first term of each tile, then the end
  for (size_t t0 = 0; t0 < short_rows.size(); t0 += 32) {
    const size_t t1 = std::min(short_rows.size(), t0 + 32);
    size_t maxlen = 0;
    for (size_t r = t0; r < t1; ++r) maxlen = std::max(maxlen, short_rows[r].terms.size());
    const size_t tile = TERMS.size();
    tile_start.push_back(tile);
    TERMS.resize(tile + 32 * maxlen, 0u);
    for (size_t r = t0; r < t1; ++r) {
      const LinRow& row = short_rows[r];
      const size_t lane = r - t0;
      for (size_t k = 0; k < row.terms.size(); ++k) TERMS[tile + 32 * k + lane] = row.terms[k];
      // flags: 1 every coefficient positive; 2 also every variable 0/1 at the root
      bool pos = true, zero_one = true;
      for (uint32_t t : row.terms) {
        const int32_t v = static_cast<int32_t>(t & 0xffffu);
        pos = pos && (static_cast<int32_t>(t) >> 16) > 0;
        zero_one = zero_one && d->lb0[v] >= 0 && d->ub0[v] <= 1;
      }
      L.push_back(make_int4(row.c, static_cast<int32_t>(tile + lane),
                            static_cast<int32_t>(row.terms.size()),
                            pos ? (zero_one ? 3 : 1) : 0));
    }
  }
  tile_start.push_back(TERMS.size());
  for (const LinRow& row : long_rows) {
    bool pos = true, zero_one = true;  // flags as for short rows
    for (uint32_t t : row.terms) {
      const int32_t v = static_cast<int32_t>(t & 0xffffu);
      pos = pos && (static_cast<int32_t>(t) >> 16) > 0;
      zero_one = zero_one && d->lb0[v] >= 0 && d->ub0[v] <= 1;
    }
    LL.push_back(make_int4(row.c, static_cast<int32_t>(TERMS_LONG.size()),
                           static_cast<int32_t>(row.terms.size()),
                           pos ? (zero_one ? 3 : 1) : 0));
    TERMS_LONG.insert(TERMS_LONG.end(), row.terms.begin(), row.terms.end());
  }
  // variable -> linear rows holding it (short rows 0.., long rows |L|..),
  // used to mark the rows to run again after the variable changes
  std::vector<std::vector<int32_t>> by_var(nv);
  auto add_row = [&by_var](const std::vector<uint32_t>& terms, int32_t r) {
    for (uint32_t t : terms) {
      std::vector<int32_t>& rows = by_var[t & 0xffffu];
      if (rows.empty() || rows.back() != r) rows.push_back(r);
    }
  };
  for (size_t r = 0; r < short_rows.size(); ++r)
    add_row(short_rows[r].terms, static_cast<int32_t>(r));
  for (size_t r = 0; r < long_rows.size(); ++r)
    add_row(long_rows[r].terms, static_cast<int32_t>(short_rows.size() + r));
  std::vector<int32_t> ADJ_OFF(nv + 1, 0), ADJ;
  for (int64_t v = 0; v < nv; ++v) {
    ADJ.insert(ADJ.end(), by_var[v].begin(), by_var[v].end());
    ADJ_OFF[v + 1] = static_cast<int32_t>(ADJ.size());
  }
  // static features of the branch variables (learned strategy)
  std::vector<BranchStatic> BST(d->n_branch);
  {
    std::vector<float> out_deg(nv, 0.f), sum_d(nv, 0.f), in_deg(nv, 0.f), n_rf(nv, 0.f);
    // demand: for the x of each reified row b <=> (x <= y < x + d), the
    // linear rows holding b with a positive bound add coef / bound; the
    // feature is the mean over those reified rows (for a scheduling start
    // variable s_i: the sum over resources of r_{k,i} / c_k)
    std::vector<double> dem_b(nv, 0.0), dem_acc(nv, 0.0);
    std::vector<int32_t> dem_cnt(nv, 0);
    for (int32_t i = 0; i < d->n_linear; ++i) {
      if (d->linear_c[i] <= 0) continue;
      for (int32_t k = d->linear_off[i]; k < d->linear_off[i + 1]; ++k)
        if (d->term_coef[k] > 0)
          dem_b[d->term_var[k]] += static_cast<double>(d->term_coef[k]) / d->linear_c[i];
    }
    for (int32_t i = 0; i < d->n_reified; ++i) {
      dem_acc[d->reified[4 * i + 1]] += dem_b[d->reified[4 * i]];
      dem_cnt[d->reified[4 * i + 1]] += 1;
    }
    for (int32_t i = 0; i < d->n_temporal; ++i) {
      out_deg[d->temporal[3 * i]] += 1.f;
      sum_d[d->temporal[3 * i]] += static_cast<float>(d->temporal[3 * i + 2]);
      in_deg[d->temporal[3 * i + 1]] += 1.f;
    }
    for (int32_t i = 0; i < d->n_reified; ++i) {
      n_rf[d->reified[4 * i + 1]] += 1.f;
      if (d->reified[4 * i + 2] != d->reified[4 * i + 1]) n_rf[d->reified[4 * i + 2]] += 1.f;
    }
    for (int32_t k = 0; k < d->n_branch; ++k) {
      const int32_t v = d->branch_vars[k];
      BranchStatic bsk;
      std::memset(&bsk, 0, sizeof(bsk));
      bsk.out_deg = out_deg[v];
      bsk.sum_d = sum_d[v];
      bsk.in_deg = in_deg[v];
      bsk.n_reified = n_rf[v];
      bsk.demand = dem_cnt[v] ? static_cast<float>(dem_acc[v] / dem_cnt[v]) : 0.f;
      BST[k] = bsk;
    }
  }

  // temporal rows in topological levels, when they form an acyclic graph:
  // the level of variable v is the length of the longest chain of rows
  // ending at v; rows are grouped by the level of their x.  Within a level no
  // row's y is another row's x, so a level's rows may run together: levels in
  // increasing order carry every lower bound along the chains in one pass,
  // in decreasing order every upper bound.
  std::vector<int32_t> TLEV_OFF;
  std::vector<uint2> TLEV;
  if (!T.empty()) {
    std::vector<int32_t> indeg(nv, 0), level(nv, 0), order;
    std::vector<std::vector<int32_t>> out(nv);
    bool acyclic = true;
    for (size_t r = 0; r < T.size(); ++r) {
      const int32_t x = static_cast<int32_t>(T[r].x & 0xffffu), y = static_cast<int32_t>(T[r].x >> 16);
      if (x == y) acyclic = false;
      out[x].push_back(static_cast<int32_t>(r));
      ++indeg[y];
    }
    for (int64_t v = 0; v < nv && acyclic; ++v)
      if (indeg[v] == 0 && !out[v].empty()) order.push_back(static_cast<int32_t>(v));
    size_t done_rows = 0;
    for (size_t q = 0; q < order.size() && acyclic; ++q) {
      const int32_t v = order[q];
      for (int32_t r : out[v]) {
        const int32_t y = static_cast<int32_t>(T[r].x >> 16);
        level[y] = std::max(level[y], level[v] + 1);
        ++done_rows;
        if (--indeg[y] == 0 && !out[y].empty()) order.push_back(y);
      }
    }
    if (acyclic && done_rows == T.size()) {
      int32_t n_lev = 0;
      for (const uint2& row : T) n_lev = std::max(n_lev, level[row.x & 0xffffu] + 1);
      TLEV_OFF.assign(n_lev + 1, 0);
      for (const uint2& row : T) ++TLEV_OFF[level[row.x & 0xffffu] + 1];
      for (int32_t l = 0; l < n_lev; ++l) TLEV_OFF[l + 1] += TLEV_OFF[l];
      std::vector<int32_t> fill(TLEV_OFF.begin(), TLEV_OFF.end() - 1);
      TLEV.resize(T.size());
      for (const uint2& row : T) TLEV[fill[level[row.x & 0xffffu]]++] = row;
    }
  }

  TableHeader h;
  std::memset(&h, 0, sizeof(h));
  h.n_vars = static_cast<int32_t>(nv);
  // store layout: Booleans from bit0 on kept as bits (bit_vars), 32 a slot
  h.bit0 = (bit0 >= 0 && bit0 < nv) ? bit0 : static_cast<int32_t>(nv);
  h.n_slots = h.bit0 + static_cast<int32_t>((nv - h.bit0 + 31) / 32);
  h.n_t = static_cast<int32_t>(T.size());
  h.n_rf = static_cast<int32_t>(RF.size());
  h.n_rfp = static_cast<int32_t>(RFP.size());
  h.n_lin = static_cast<int32_t>(L.size());
  h.n_lin_long = static_cast<int32_t>(LL.size());
  h.n_terms = n_terms;
  h.n_branch = d->n_branch;
  h.objective = d->objective;
  h.rows_sweep = h.n_t + h.n_rf + 2 * h.n_rfp + h.n_lin + h.n_lin_long;
  if (bytes_per_sweep > static_cast<int64_t>(INT32_MAX)) return PCCP_ERR_UNSUPPORTED;
  h.bytes_sweep = static_cast<int32_t>(bytes_per_sweep);
  size_t off = sizeof(TableHeader);
  h.off_t = static_cast<int32_t>(off);
  off = align16(off + T.size() * sizeof(uint2));
  h.off_rf = static_cast<int32_t>(off);
  off = align16(off + RF.size() * sizeof(uint2));
  h.off_rfp = static_cast<int32_t>(off);
  off = align16(off + RFP.size() * sizeof(uint4));
  h.off_lin = static_cast<int32_t>(off);
  off = align16(off + L.size() * sizeof(int4));
  h.off_terms = static_cast<int32_t>(off);
  off = align16(off + TERMS.size() * sizeof(uint32_t));
  h.off_lin_long = static_cast<int32_t>(off);
  off = align16(off + LL.size() * sizeof(int4));
  h.off_terms_long = static_cast<int32_t>(off);
  off = align16(off + TERMS_LONG.size() * sizeof(uint32_t));
  h.off_branch = static_cast<int32_t>(off);
  off = align16(off + static_cast<size_t>(d->n_branch) * sizeof(int32_t));
  h.off_bstat = static_cast<int32_t>(off);
  off = align16(off + BST.size() * sizeof(BranchStatic));
  h.off_tlev = static_cast<int32_t>(off);
  h.n_tlev = TLEV_OFF.empty() ? 0 : static_cast<int32_t>(TLEV_OFF.size()) - 1;
  off = align16(off + TLEV_OFF.size() * sizeof(int32_t));
  off = align16(off + TLEV.size() * sizeof(uint2));
  h.core_bytes = static_cast<int32_t>(off);  // what the eventless kernels copy
  h.off_adj_off = static_cast<int32_t>(off);
  off = align16(off + ADJ_OFF.size() * sizeof(int32_t));
  h.off_adj = static_cast<int32_t>(off);
  h.n_adj = static_cast<int32_t>(ADJ.size());
  off = align16(off + ADJ.size() * sizeof(int32_t));
  h.track_bytes = static_cast<int32_t>(off);  // ... and the kernels that skip stable rows
  // Stream segments: the row sections cut into byte ranges of whole rows of
  // at most kStreamChunk bytes, 16-byte aligned (a range may run into the
  // section's padding), in the order a sweep evaluates them.
  std::vector<StreamSeg> SEG;
  auto seg = [&SEG](int32_t kind, size_t first, size_t count, size_t src, size_t bytes,
                    size_t term_base) {
    StreamSeg s;
    std::memset(&s, 0, sizeof(s));
    s.kind = kind;
    s.first = static_cast<int32_t>(first);
    s.count = static_cast<int32_t>(count);
    s.src_off = static_cast<int32_t>(src);
    s.bytes = static_cast<int32_t>(bytes);
    s.term_base = static_cast<int32_t>(term_base);
    SEG.push_back(s);
  };
  auto fixed_rows = [&seg](int32_t kind, size_t n, size_t rec, size_t section) {
    const size_t per = kStreamChunk / rec;
    for (size_t f = 0; f < n; f += per) {
      const size_t c = std::min(per, n - f);
      seg(kind, f, c, section + f * rec, align16(c * rec), 0);
    }
  };
  fixed_rows(kSegPairs, RFP.size(), sizeof(uint4), static_cast<size_t>(h.off_rfp));
  fixed_rows(kSegSingles, RF.size(), sizeof(uint2), static_cast<size_t>(h.off_rf));
  fixed_rows(kSegTemporal, T.size(), sizeof(uint2), static_cast<size_t>(h.off_t));
  const size_t n_tiles = tile_start.size() - 1;
  for (size_t t0 = 0; t0 < n_tiles;) {  // whole tiles (a tile is at most 8 KB)
    size_t t1 = t0 + 1;
    while (t1 < n_tiles && 4 * (tile_start[t1 + 1] - tile_start[t0]) <= kStreamChunk) ++t1;
    const size_t rows = std::min(L.size(), 32 * t1) - 32 * t0;
    seg(kSegShort, 32 * t0, rows, h.off_terms + 4 * tile_start[t0],
        4 * (tile_start[t1] - tile_start[t0]), tile_start[t0]);
    t0 = t1;
  }
  for (size_t r0 = 0; r0 < LL.size();) {  // whole long rows
    const size_t start = (4 * static_cast<size_t>(LL[r0].y)) & ~static_cast<size_t>(15);
    auto end_of = [&LL](size_t r) { return align16(4 * static_cast<size_t>(LL[r].y + LL[r].z)); };
    if (end_of(r0) - start > static_cast<size_t>(kStreamChunk)) {
      seg(kSegLongGlobal, r0, 1, 0, 0, 0);  // longer than a chunk: read in place
      ++r0;
      continue;
    }
    size_t r1 = r0 + 1;
    while (r1 < LL.size() && end_of(r1) - start <= static_cast<size_t>(kStreamChunk)) ++r1;
    seg(kSegLong, r0, r1 - r0, h.off_terms_long + start, end_of(r1 - 1) - start, start / 4);
    r0 = r1;
  }
  h.off_seg = static_cast<int32_t>(off);
  h.n_seg = static_cast<int32_t>(SEG.size());
  off = align16(off + SEG.size() * sizeof(StreamSeg));
  if (off > (1u << 30)) return PCCP_ERR_UNSUPPORTED;
  h.image_bytes = static_cast<int32_t>(off);

  p->image.assign(off, 0);
  std::memcpy(p->image.data(), &h, sizeof(h));
  if (!T.empty()) std::memcpy(p->image.data() + h.off_t, T.data(), T.size() * sizeof(uint2));
  if (!RF.empty()) std::memcpy(p->image.data() + h.off_rf, RF.data(), RF.size() * sizeof(uint2));
  if (!RFP.empty())
    std::memcpy(p->image.data() + h.off_rfp, RFP.data(), RFP.size() * sizeof(uint4));
  if (!L.empty()) std::memcpy(p->image.data() + h.off_lin, L.data(), L.size() * sizeof(int4));
  if (!TERMS.empty())
    std::memcpy(p->image.data() + h.off_terms, TERMS.data(), TERMS.size() * sizeof(uint32_t));
  if (!LL.empty()) std::memcpy(p->image.data() + h.off_lin_long, LL.data(), LL.size() * sizeof(int4));
  if (!TERMS_LONG.empty())
    std::memcpy(p->image.data() + h.off_terms_long, TERMS_LONG.data(),
                TERMS_LONG.size() * sizeof(uint32_t));
  if (d->n_branch > 0)
    std::memcpy(p->image.data() + h.off_branch, d->branch_vars,
                static_cast<size_t>(d->n_branch) * sizeof(int32_t));
  std::memcpy(p->image.data() + h.off_adj_off, ADJ_OFF.data(), ADJ_OFF.size() * sizeof(int32_t));
  if (!ADJ.empty())
    std::memcpy(p->image.data() + h.off_adj, ADJ.data(), ADJ.size() * sizeof(int32_t));
  if (!BST.empty())
    std::memcpy(p->image.data() + h.off_bstat, BST.data(), BST.size() * sizeof(BranchStatic));
  if (!SEG.empty())
    std::memcpy(p->image.data() + h.off_seg, SEG.data(), SEG.size() * sizeof(StreamSeg));
  if (!TLEV.empty()) {
    std::memcpy(p->image.data() + h.off_tlev, TLEV_OFF.data(), TLEV_OFF.size() * sizeof(int32_t));
    std::memcpy(p->image.data() + align16(h.off_tlev + TLEV_OFF.size() * sizeof(int32_t)),
                TLEV.data(), TLEV.size() * sizeof(uint2));
  }
  p->n_vars = h.n_vars;
  p->n_t = h.n_t;
  p->n_rf = h.n_rf + 2 * h.n_rfp;
  p->n_lin = h.n_lin + h.n_lin_long;
  p->n_terms = h.n_terms;
  p->n_branch = h.n_branch;
  p->objective = h.objective;
  p->bytes_per_sweep = bytes_per_sweep;
  p->n_seg = h.n_seg;
  p->core_bytes = static_cast<uint32_t>(h.core_bytes);
  p->track_bytes = static_cast<uint32_t>(h.track_bytes);
  p->bit0 = h.bit0;
  p->n_slots = h.n_slots;
  p->n_tlev = h.n_tlev;
  p->tlev_bytes = static_cast<uint32_t>(h.core_bytes - h.off_tlev);
  return PCCP_OK;
}

// Shared memory of k_solve: table image, mbarrier, control, change
// tracking, one store.
size_t solve_smem(uint32_t max_img, int max_track_words, int max_vars, int x_words = 0) {
  return static_cast<size_t>(max_img) + 16 + sizeof(SearchCtrl) +
         4 * static_cast<size_t>((max_track_words + 3) & ~3) +
         static_cast<size_t>(max_vars) * sizeof(int2) + 4 * static_cast<size_t>(x_words);
}

// Stream buffers per team for a table read from global memory: the most
// (3, else 2) that fit beside `teams` teams of `per_team` bytes; 0 when the
// table has no rows, streaming is not asked for, or not even two fit.
int stream_stages_for(int n_seg, int stream_opt, size_t fixed, size_t per_team, int teams,
                      int smem_max) {
  if (n_seg <= 0 || stream_opt <= 0) return 0;
  for (int s = kStreamMaxStages; s >= 2; --s)
    if (fixed + static_cast<size_t>(teams) * (per_team + stream_bytes(s)) <=
        static_cast<size_t>(smem_max))
      return s;
  return 0;
}

// Shared memory of k_solve, with the tables in shared memory when they fit,
// else read from the device images (*global = true), streamed through
// *stages buffers when the largest segment list is non-empty and they fit.
size_t plan_solve_smem(uint32_t max_img, int max_track_words, int max_vars, int smem_max,
                       bool* global, int x_words, int stream_opt, int max_seg, int* stages) {
  const size_t with = solve_smem(max_img, max_track_words, max_vars, x_words);
  *global = with > static_cast<size_t>(smem_max);
  *stages = 0;
  if (!*global) return with;
  const size_t base = solve_smem(0, max_track_words, max_vars, x_words);
  *stages = stream_stages_for(max_seg, stream_opt, base, 0, 1, smem_max);
  return base + stream_bytes(*stages);
}

// Words of shared memory for the learned strategy's feature rows (0 otherwise).
int policy_x_words(const pccp_solve_opts* o, int max_branch) {
  return o->strategy == PCCP_LEARNED ? 24 * ((max_branch + 15) & ~15) : 0;
}

// skip_stable of the launch options: 1 on, -1 off, 0 the library's choice --
// on for tables read from global memory (many iterations over a large table:
// measured 17% faster on 120-task models), off for tables in shared memory
// (the change bitmaps cost more than the rows they save there).
bool use_skip_stable(int32_t opt, bool global) { return opt > 0 || (opt == 0 && global); }

// The one-team kernel that streams the tables through shared memory (a
// batched search that asks for streaming when some table does not fit).
using SolveKernel = void (*)(SolveArgs);
SolveKernel stream_kernel(const pccp_solve_opts* o) {
  if (o->strategy == PCCP_LEARNED) return k_solve<false, true, true, true>;
  return use_skip_stable(o->skip_stable, true) ? k_solve<true, false, true, true>
                                               : k_solve<false, false, true, true>;
}

// The k_solve_slots instantiation for a search's options: change tracking
// for tables staged in shared memory / read from global memory.
SolveKernel slots_kernel(const pccp_solve_opts* o) {
  if (o->strategy == PCCP_LEARNED) return k_solve_slots<false, false, true>;
  if (o->skip_stable > 0) return k_solve_slots<true, true, false>;
  if (o->skip_stable < 0) return k_solve_slots<false, false, false>;
  return k_solve_slots<false, true, false>;
}

// Strategy and policy checks shared by the search entry points.
int check_strategy(const pccp_solve_opts* o) {
  if (o->strategy != PCCP_INPUT_ORDER && o->strategy != PCCP_FIRST_FAIL &&
      o->strategy != PCCP_LEARNED)
    return PCCP_ERR_INVALID;
  if (o->mode != PCCP_OPTIMISE && o->mode != PCCP_COUNT_ALL) return PCCP_ERR_INVALID;
  if (o->strategy == PCCP_LEARNED) {
    if (!o->policy) return PCCP_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PCCP_ERR_CUDA;
    if (dev != policy_device(o->policy)) return PCCP_ERR_INVALID;
  }
  return PCCP_OK;
}

int max_dyn_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return -1;
  return v;
}

int sm_count() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  return v;
}

// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `smem`.  Limits only grow, so a plan made on another host thread for
// a smaller model cannot lower the limit between this plan and its launch.
cudaError_t allow_smem(const void* kern, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<uint64_t, std::unordered_map<const void*, size_t>> set;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = set[static_cast<uint64_t>(dev)][kern];
  if (cur >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
  if (e == cudaSuccess) cur = smem;
  return e;
}

int check_device(const pccp_model* m) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PCCP_ERR_CUDA;
  return dev == m->device ? PCCP_OK : PCCP_ERR_INVALID;
}

#define PCCP_CUDA(call)                    \
  do {                                     \
    if ((call) != cudaSuccess) {           \
      (void)cudaGetLastError();            \
      return PCCP_ERR_CUDA;                \
    }                                      \
  } while (0)

struct PropPlan {
  void (*kern)(PropArgs);
  bool table_global;
  uint32_t copy_bytes;  // image prefix staged in shared memory (0: read in place)
  int stages;  // stream buffers per team (0: rows read in place)
  uint32_t tlev_bytes;  // rows read in place: the temporal levels staged per CTA (0: none)
  int team, teams, grid, max_grid;
  size_t smem;
};

int plan_propagate(const pccp_model* m, int32_t n_stores, const pccp_launch_config* cfg,
                   PropPlan* p) {
  const int smem_max = max_dyn_smem();
  const int sms = sm_count();
  if (smem_max <= 0 || sms <= 0) return PCCP_ERR_CUDA;
  int team = (cfg && cfg->team_threads > 0) ? cfg->team_threads : 128;
  if (team % 32 != 0 || team > 1024) return PCCP_ERR_INVALID;
  const size_t per_team = sizeof(PropCtrl) + 4 * ((track_words(m->n_vars, m->n_lin) + 3) & ~3) +
                          static_cast<size_t>(m->n_slots) * sizeof(int2);
  // the table lives in shared memory when it fits beside one team's store
  // (the prefix the kernel needs: with change tracking, the adjacency too);
  // otherwise every CTA reads it from the device image (through L1 / L2)
  const uint32_t img_smem =
      use_skip_stable(cfg ? cfg->skip_stable : 0, false) ? m->track_bytes : m->core_bytes;
  const bool bits = m->bit0 < m->n_vars;  // read only by the global-table kernels
  const bool global = bits || static_cast<size_t>(img_smem) + 16 + per_team >
                                  static_cast<size_t>(smem_max);
  const size_t base = (global ? 0 : static_cast<size_t>(img_smem)) + 16;
  if (base + per_team > static_cast<size_t>(smem_max)) return PCCP_ERR_SMEM;
  if (global && !(cfg && cfg->team_threads > 0)) team = 1024;
  int fit = static_cast<int>((static_cast<size_t>(smem_max) - base) / per_team);
  // default: 8 teams of 128 threads per CTA, one CTA per SM (32 warps of up
  // to 64 registers; measured ahead of 4 x 128 with three CTAs per SM and a
  // 40-register cap)
  int teams = (cfg && cfg->teams_per_cta > 0) ? cfg->teams_per_cta : 8;
  if (teams > kMaxTeamsPerCta) return PCCP_ERR_INVALID;
  teams = std::min({teams, fit, 1024 / team});
  if (cfg && cfg->teams_per_cta > 0 && teams < cfg->teams_per_cta) return PCCP_ERR_SMEM;
  if (teams < 1) return PCCP_ERR_SMEM;
  const int stages = global ? stream_stages_for(m->n_seg, cfg ? cfg->stream_table : 0, base,
                                                per_team, teams, smem_max)
                            : 0;
  size_t smem = base + static_cast<size_t>(teams) * (per_team + stream_bytes(stages));
  // rows read in place: the temporal rows' levels (a few KB) staged once per
  // CTA when they fit, since their passes are chains of dependent loads
  uint32_t tlev = 0;
  if (global && stages == 0 && m->n_tlev > 0 &&
      (levels_mask(cfg ? cfg->temporal_levels : 0, true) & 2) &&
      smem + m->tlev_bytes <= static_cast<size_t>(smem_max)) {
    tlev = m->tlev_bytes;
    smem += tlev;
  }
  const bool track = use_skip_stable(cfg ? cfg->skip_stable : 0, global);
  const auto kern =
      stages > 0 ? (track ? k_propagate<1024, 1, true, true, true>
                          : k_propagate<1024, 1, false, true, true>)
      : global   ? (track ? k_propagate<1024, 1, true, true, false>
                          : k_propagate<1024, 1, false, true, false>)
      : (teams * team <= 512)
          ? (track ? k_propagate<512, 3, true, false, false>
                   : k_propagate<512, 3, false, false, false>)
          : (track ? k_propagate<1024, 1, true, false, false>
                   : k_propagate<1024, 1, false, false, false>);
  if (allow_smem(reinterpret_cast<const void*>(kern), smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return PCCP_ERR_CUDA;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, teams * team, smem) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return PCCP_ERR_CUDA;
  }
  if (per_sm < 1) return PCCP_ERR_SMEM;
  if (cfg && cfg->ctas_per_sm > 0) per_sm = std::min(per_sm, static_cast<int>(cfg->ctas_per_sm));
  const int want = (n_stores + teams - 1) / teams;
  p->kern = kern;
  p->table_global = global;
  p->copy_bytes = global ? 0u : img_smem;
  p->stages = stages;
  p->tlev_bytes = tlev;
  p->team = team;
  p->teams = teams;
  p->max_grid = sms * per_sm;
  p->grid = std::max(1, std::min(want, p->max_grid));
  p->smem = smem;
  return PCCP_OK;
}

// Queue one k_propagate launch of a plan over n_stores stores (>= 1), with
// counter a zeroed device int; the grid shrinks for batches smaller than the
// one planned.
int launch_propagate(const pccp_model* m, const PropPlan& plan, int32_t n_stores, int32_t* lb,
                     int32_t* ub, int32_t* status, int32_t* iterations, int32_t* work,
                     const pccp_launch_config* cfg, int* counter, cudaStream_t s) {
  PropArgs a;
  a.image = m->d_mem;
  a.root = m->d_root;
  a.lb = lb;
  a.ub = ub;
  a.status = status;
  a.iters = iterations;
  a.counter = counter;
  a.image_bytes = plan.table_global ? m->image_bytes : plan.copy_bytes;
  a.n_vars = m->n_vars;
  a.n_slots = m->n_slots;
  a.n_stores = n_stores;
  a.team_size = plan.team;
  a.teams = plan.teams;
  a.max_iter = (cfg && cfg->max_iterations > 0) ? cfg->max_iterations : m->max_iter;
  a.track_words = track_words(m->n_vars, m->n_lin);
  a.work = work;
  a.table_global = plan.table_global ? 1 : 0;
  a.stream_stages = plan.stages;
  a.reordered = m->reordered;
  a.tlev_bytes = plan.tlev_bytes;
  a.levels = levels_mask(cfg ? cfg->temporal_levels : 0, true);
  a.off_tlev = m->core_bytes - m->tlev_bytes;
  const int grid = std::max(1, std::min((n_stores + plan.teams - 1) / plan.teams, plan.max_grid));
  plan.kern<<<grid, plan.team * plan.teams, plan.smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? PCCP_OK : PCCP_ERR_CUDA;
}

// Launch plan of a batched search (pccp_solve_batch, pccp_batch_*,
// pccp_solve_batch_noalloc).
struct BatchPlan {
  SolveKernel kern;
  bool slots;            // k_solve_slots; else the one-team streamed kernel
  int team, teams, grid, max_depth;
  size_t smem;           // dynamic shared memory per CTA
  uint32_t slot_bytes, off_track, off_x, off_stack, off_store;
  int xw, max_tw, max_vars, stages;
};

// Shared memory a model needs in a slot whose store starts at off_store:
// the store, then its table prefix 128-byte aligned (when `staged`).
uint32_t slot_need(const pccp_model* m, uint32_t off_store, bool track, bool staged) {
  const uint32_t st_end = off_store + 8u * static_cast<uint32_t>(m->n_slots);
  if (!staged || m->bit0 < m->n_vars) return st_end;  // bit layouts are read in place
  return ((st_end + 127u) & ~127u) + (track ? m->track_bytes : m->core_bytes);
}

// Slot bytes of a model whose table is read in place, with its temporal
// levels staged after the store when that fits in `room` (else without).
uint32_t slot_need_global(const pccp_model* m, uint32_t off_store, uint32_t room) {
  const uint32_t st_end = off_store + 8u * static_cast<uint32_t>(m->n_slots);
  const uint32_t with = ((st_end + 127u) & ~127u) + m->tlev_bytes;
  return m->n_tlev > 0 && with <= room ? with : st_end;
}

// Plans a batched search.  any_strategy: room for the learned strategy's
// feature rows and an occupancy valid for every strategy's kernel (a batch
// planned once for later searches).  Returns SMEM when some store does not
// fit a slot.
int plan_batch(const pccp_model* const* models, int32_t n, const pccp_solve_opts* o,
               bool any_strategy, BatchPlan* p) {
  const int smem_max = max_dyn_smem();
  const int sms = sm_count();
  if (smem_max <= 0 || sms <= 0) return PCCP_ERR_CUDA;
  int32_t max_vars = 0, max_branch = 0, max_tw = 0, max_seg = 0, max_rows = 0, max_dec = 2;
  uint32_t max_core = 0;
  for (int32_t i = 0; i < n; ++i) {
    const pccp_model* m = models[i];
    max_dec = std::max(max_dec, m->max_decisions);
    max_vars = std::max(max_vars, m->n_slots);  // store slots
    max_branch = std::max(max_branch, m->n_branch);
    max_tw = std::max(max_tw, track_words(m->n_vars, m->n_lin));
    max_seg = std::max(max_seg, m->n_seg);
    max_rows = std::max(max_rows, m->n_t + m->n_rf + m->n_lin);
    max_core = std::max(max_core, m->core_bytes);
  }
  if (o->threads < 0 || o->threads % 32 != 0 || o->threads > 1024) return PCCP_ERR_INVALID;
  if (o->teams_per_cta < 0 || o->teams_per_cta > kMaxTeamsPerCta) return PCCP_ERR_INVALID;
  if (o->props_per_thread < 0) return PCCP_ERR_INVALID;
  p->xw = any_strategy ? 24 * ((max_branch + 15) & ~15) : policy_x_words(o, max_branch);
  p->max_tw = max_tw;
  p->max_vars = max_vars;
  p->max_depth = max_dec;
  p->off_track = static_cast<uint32_t>(align16(16 + sizeof(SearchCtrl)));
  p->off_x = p->off_track + 4u * static_cast<uint32_t>((max_tw + 3) & ~3);
  p->off_stack = static_cast<uint32_t>(align16(p->off_x + 4u * static_cast<uint32_t>(p->xw)));
  p->off_store = static_cast<uint32_t>(
      align16(p->off_stack + sizeof(int2) * static_cast<size_t>(p->max_depth)));
  const bool track_s = o->strategy != PCCP_LEARNED && o->skip_stable > 0;
  // streaming (one team per CTA, the old kernel) only when asked for and some
  // table prefix does not fit one CTA beside its store
  bool all_fit_one = true;
  for (int32_t i = 0; i < n; ++i)
    all_fit_one = all_fit_one && slot_need(models[i], p->off_store, track_s, true) <=
                                     static_cast<uint32_t>(smem_max);
  if (o->stream_table > 0 && !all_fit_one && !any_strategy) {
    bool global = false;
    int stages = 0;
    const size_t smem = plan_solve_smem(max_core, max_tw, max_vars, smem_max, &global, p->xw,
                                        o->stream_table, max_seg, &stages);
    if (global && stages > 0) {
      if (smem > static_cast<size_t>(smem_max)) return PCCP_ERR_SMEM;
      p->slots = false;
      p->kern = stream_kernel(o);
      p->team = o->threads > 0 ? o->threads : 1024;
      p->teams = 1;
      p->smem = smem;
      p->stages = stages;
      p->slot_bytes = p->off_track = p->off_x = p->off_stack = p->off_store = 0;
      PCCP_CUDA(allow_smem(reinterpret_cast<const void*>(p->kern), smem));
      int per_sm = 0;
      PCCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->kern, p->team, smem));
      if (per_sm < 1) return PCCP_ERR_SMEM;
      p->grid = std::max(1, std::min(n, sms * per_sm));
      if (o->blocks > 0) p->grid = std::min(p->grid, static_cast<int>(o->blocks));
      return PCCP_OK;
    }
  }
  p->slots = true;
  p->stages = 0;
  p->kern = slots_kernel(o);
  // teams per CTA: asked for, else the most slots (up to 8) in which every
  // model's table fits beside its store, else one
  int teams = o->teams_per_cta;
  if (teams == 0) {
    teams = 1;
    const int k_max = std::min(8, 1024 / std::max(o->threads, 32));
    for (int k = k_max; k >= 2; --k) {
      const uint32_t room = static_cast<uint32_t>(smem_max / k) & ~127u;
      bool fit = true;
      for (int32_t i = 0; fit && i < n; ++i)
        fit = slot_need(models[i], p->off_store, track_s, true) <= room;
      if (fit) {
        teams = k;
        break;
      }
    }
  }
  int team = o->threads;
  if (team == 0 && o->props_per_thread > 0)
    team = std::min(1024 / teams, std::max(32, ((max_rows + o->props_per_thread - 1) /
                                                    o->props_per_thread + 31) & ~31));
  // default team: 256 threads when several share a CTA; a whole CTA when one
  // team has it (its search is a chain of dependent sweeps, which the lane
  // groups of the linear rows shorten with more lanes: 256 30-60-task models
  // x 4,000 nodes in 353 ms at 1024 threads, 370 at 512, 401 at 256)
  if (team == 0)
    team = all_fit_one && teams > 1 ? std::min(256, (1024 / teams) & ~31) : (1024 / teams) & ~31;
  if (team < 32 || team * teams > 1024) return PCCP_ERR_INVALID;
  // slot size: what the largest model needs (staged when it fits), at most
  // an equal share of the CTA's shared memory
  const uint32_t room = static_cast<uint32_t>(smem_max / teams) & ~127u;
  uint32_t want = 0;
  for (int32_t i = 0; i < n; ++i) {
    const uint32_t staged = slot_need(models[i], p->off_store, track_s, true);
    const uint32_t need =
        staged <= room ? staged : slot_need_global(models[i], p->off_store, room);
    want = std::max(want, need);
  }
  if (want > room) return PCCP_ERR_SMEM;  // a store alone does not fit
  p->slot_bytes = (want + 127u) & ~127u;
  p->team = team;
  p->teams = teams;
  p->smem = static_cast<size_t>(teams) * p->slot_bytes;
  // (a fixed array: the allocation-free entry point plans with this too)
  SolveKernel kerns[8] = {p->kern};
  int n_kerns = 1;
  if (any_strategy) {
    pccp_solve_opts q = *o;
    for (int strategy : {PCCP_INPUT_ORDER, PCCP_LEARNED})
      for (int skip : {-1, 0, 1}) {
        q.strategy = strategy;
        q.skip_stable = skip;
        if (n_kerns < 8) kerns[n_kerns++] = slots_kernel(&q);
      }
  }
  int per_sm = 1 << 30;
  for (int ki = 0; ki < n_kerns; ++ki) {
    const SolveKernel k = kerns[ki];
    PCCP_CUDA(allow_smem(reinterpret_cast<const void*>(k), p->smem));
    int occ = 0;
    PCCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, team * teams, p->smem));
    per_sm = std::min(per_sm, occ);
  }
  if (per_sm < 1) return PCCP_ERR_SMEM;
  // one CTA per model up to the resident limit: models spread over the SMs
  // before teams share one (a team's search is a chain of dependent nodes,
  // so a model alone on an SM finishes first)
  p->grid = std::max(1, std::min(static_cast<int>(n), sms * per_sm));
  if (o->blocks > 0) p->grid = std::min(p->grid, static_cast<int>(o->blocks));
  return PCCP_OK;
}

// Queue order of a batch: largest table first (ties by position), so the
// longest searches start first and the small ones fill the tail.
std::vector<int32_t> batch_order(const pccp_model* const* models, int32_t n) {
  std::vector<int32_t> ord(n);
  for (int32_t i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [models](int32_t a, int32_t b) {
    return models[a]->image_bytes > models[b]->image_bytes;
  });
  return ord;
}

// Descriptor of model i (position `index` in the caller's list).
InstanceDesc instance_desc(const pccp_model* m, int32_t index, int32_t witness_off) {
  InstanceDesc d;
  d.image = m->d_mem;
  d.root = m->d_root;
  d.image_bytes = m->image_bytes;
  d.n_vars = m->n_vars;
  d.witness_off = witness_off;
  d.n_branch = m->n_branch;
  d.max_iter = m->max_iter;
  d.index = index;
  return d;
}

// Kernel arguments of a planned batched search (buffers filled by the caller).
SolveArgs batch_args(const BatchPlan& p, const pccp_solve_opts* o, int32_t n) {
  SolveArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_inst = n;
  a.max_depth = p.max_depth;
  a.mode = o->mode;
  a.strategy = o->strategy;
  a.obj_ub = o->obj_ub;
  a.levels = levels_mask(o->temporal_levels, false);
  a.node_limit = o->node_limit;
  a.time_limit_ns = o->time_limit_ms > 0 ? o->time_limit_ms * 1000000ll : 0;
  a.max_image_bytes = 0;  // the streamed kernel reads every table from global memory
  a.max_track_words = p.max_tw;
  a.table_global = 1;
  a.stream_stages = p.stages;
  a.x_words = p.xw;
  a.max_vars_smem = p.max_vars;
  a.policy = o->strategy == PCCP_LEARNED ? policy_dev(o->policy) : nullptr;
  a.team_size = p.team;
  a.teams = p.teams;
  a.slot_bytes = p.slot_bytes;
  a.off_track = p.off_track;
  a.off_x = p.off_x;
  a.off_stack = p.off_stack;
  a.off_store = p.off_store;
  return a;
}

// Parallel search over a shared queue of subproblems (defined with the
// parallel search entry points below).
int solve_queue(const pccp_model* const* models, int32_t n, const pccp_solve_opts* o,
                pccp_result* results, cudaStream_t s);

}  // namespace

extern "C" {

const char* pccp_error_string(int code) {
  switch (code) {
    case PCCP_OK: return "ok";
    case PCCP_ERR_INVALID: return "invalid argument";
    case PCCP_ERR_OVERFLOW: return "a propagator intermediate could overflow int32";
    case PCCP_ERR_SMEM: return "model does not fit in shared memory";
    case PCCP_ERR_TIMEOUT: return "a device wait or iteration budget ran out";
    case PCCP_ERR_CUDA: return "CUDA runtime error";
    case PCCP_ERR_UNSUPPORTED: return "model outside the packed-table limits";
    case PCCP_ERR_SCRATCH: return "request exceeds the fixed scratch of the allocation-free call";
    default: return "unknown error";
  }
}

int pccp_model_create(const pccp_model_desc* desc_user, pccp_model** out) {
  if (!out) return PCCP_ERR_INVALID;
  *out = nullptr;
  if (!desc_user) return PCCP_ERR_INVALID;
  const int32_t nv_user = desc_user->n_vars > 0 ? desc_user->n_vars : 0;
  // Booleans kept as bits when the model allows it (bit_vars) and either the
  // caller asks for it or an interval store would exceed kBitStoreMinBytes
  std::vector<char> bits;
  int32_t n_bits = 0;
  if (desc_user->bool_store >= 0) {
    bits = bit_vars(desc_user);
    for (char b : bits) n_bits += b ? 1 : 0;
    // by default only where an interval store could not fit in shared memory
    // at all (the model would be refused): bits cost an extraction per
    // Boolean read and are read only by the global-table kernels, which
    // measured slower than interval stores wherever those fit
    bool want = desc_user->bool_store > 0;
    if (!want && n_bits > 0) {
      const int smem_max = max_dyn_smem();
      want = smem_max > 0 && 8ll * nv_user + kBitStoreSlack > smem_max;
    }
    if (n_bits == 0 || !want) {
      bits.clear();
      n_bits = 0;
    }
  }
  // the model in the library's variable order (internal_order / bit_order)
  const std::vector<int32_t> iof =
      bits.empty() ? internal_order(desc_user) : bit_order(desc_user, bits);
  std::vector<int32_t> uof(nv_user);
  for (int32_t v = 0; v < nv_user; ++v) uof[iof[v]] = v;
  auto map_var = [&iof, nv_user](int32_t v) { return v >= 0 && v < nv_user ? iof[v] : v; };
  std::vector<int32_t> lb0, ub0, tmp, rf, tv, br;
  pccp_model_desc dd = *desc_user;
  if (desc_user->lb0 && desc_user->ub0) {
    lb0.resize(nv_user);
    ub0.resize(nv_user);
    for (int32_t v = 0; v < nv_user; ++v) {
      lb0[iof[v]] = desc_user->lb0[v];
      ub0[iof[v]] = desc_user->ub0[v];
    }
    dd.lb0 = lb0.data();
    dd.ub0 = ub0.data();
  }
  if (desc_user->n_temporal > 0 && desc_user->temporal) {
    tmp.assign(desc_user->temporal, desc_user->temporal + 3 * desc_user->n_temporal);
    for (int32_t i = 0; i < desc_user->n_temporal; ++i) {
      tmp[3 * i] = map_var(tmp[3 * i]);
      tmp[3 * i + 1] = map_var(tmp[3 * i + 1]);
    }
    dd.temporal = tmp.data();
  }
  if (desc_user->n_reified > 0 && desc_user->reified) {
    rf.assign(desc_user->reified, desc_user->reified + 4 * desc_user->n_reified);
    for (int32_t i = 0; i < desc_user->n_reified; ++i)
      for (int k = 0; k < 3; ++k) rf[4 * i + k] = map_var(rf[4 * i + k]);
    dd.reified = rf.data();
  }
  bool offsets_ok = desc_user->n_linear > 0 && desc_user->linear_off && desc_user->term_var &&
                    desc_user->linear_off[0] == 0;
  for (int32_t i = 0; offsets_ok && i < desc_user->n_linear; ++i)
    offsets_ok = desc_user->linear_off[i + 1] >= desc_user->linear_off[i];
  if (offsets_ok) {  // else validation rejects the model before reading terms
    const int32_t nt = desc_user->linear_off[desc_user->n_linear];
    tv.assign(desc_user->term_var, desc_user->term_var + nt);
    for (int32_t& v : tv) v = map_var(v);
    dd.term_var = tv.data();
  }
  if (desc_user->n_branch > 0 && desc_user->branch_vars) {
    br.assign(desc_user->branch_vars, desc_user->branch_vars + desc_user->n_branch);
    for (int32_t& v : br) v = map_var(v);
    dd.branch_vars = br.data();
  }
  dd.objective = map_var(desc_user->objective);
  const pccp_model_desc* desc = &dd;
  Packed p;
  const int rc = validate_and_pack(desc, &p, n_bits > 0 ? nv_user - n_bits : -1);
  if (rc != PCCP_OK) return rc;
  int dev = 0;
  PCCP_CUDA(cudaGetDevice(&dev));
  pccp_model* m = new (std::nothrow) pccp_model;
  if (!m) return PCCP_ERR_INVALID;
  m->device = dev;
  m->n_vars = p.n_vars;
  m->n_t = p.n_t;
  m->n_rf = p.n_rf;
  m->n_lin = p.n_lin;
  m->n_terms = p.n_terms;
  m->n_branch = p.n_branch;
  m->objective = p.objective;
  m->image_bytes = static_cast<uint32_t>(p.image.size());
  m->core_bytes = p.core_bytes;
  m->track_bytes = p.track_bytes;
  m->n_tlev = p.n_tlev;
  m->tlev_bytes = p.tlev_bytes;
  m->bytes_per_sweep = p.bytes_per_sweep;
  m->n_seg = p.n_seg;
  m->reordered = 0;
  for (int32_t v = 0; v < nv_user; ++v) m->reordered |= iof[v] != v ? 1 : 0;
  {
    // total width of the root box + 3 bounds the iterations of any store
    int64_t w = 3;
    for (int v = 0; v < p.n_vars; ++v) w += static_cast<int64_t>(desc->ub0[v]) - desc->lb0[v];
    m->max_iter = static_cast<int32_t>(std::min<int64_t>(w, kDefaultMaxIter));
    // a split leaves at most floor(width / 2) on either side, so a branch
    // variable of root width w takes at most bitlen(w) decisions on one path
    int64_t dec = 2;
    for (int32_t k = 0; k < p.n_branch; ++k) {
      const int32_t v = desc->branch_vars[k];
      uint32_t wv = static_cast<uint32_t>(static_cast<int64_t>(desc->ub0[v]) - desc->lb0[v]);
      while (wv) {
        ++dec;
        wv >>= 1;
      }
    }
    m->max_decisions = static_cast<int32_t>(std::min<int64_t>(dec, INT32_MAX));
  }
  // device memory: image | root int2[n] | internal_of int32[n] | user_of int32[n]
  // device memory: image | root int2[n] | internal_of int32[n] | user_of
  // int32[n] | the root in the store layout int2[n_slots] (Boolean slots as
  // bit words; bits past the last Boolean: lower 0, upper 1)
  const size_t root_off = align16(p.image.size());
  const size_t total = root_off + static_cast<size_t>(p.n_vars) * (sizeof(int2) + 8) +
                       static_cast<size_t>(p.n_slots) * sizeof(int2);
  std::vector<int2> root(p.n_vars);
  for (int v = 0; v < p.n_vars; ++v) root[v] = make_int2(desc->lb0[v], desc->ub0[v]);
  std::vector<int2> root_store(p.n_slots);
  for (int v = 0; v < p.bit0; ++v) root_store[v] = root[v];
  for (int sl = p.bit0; sl < p.n_slots; ++sl) {
    uint32_t lw = 0u, uw = 0u;
    for (int j = 0; j < 32; ++j) {
      const int v = p.bit0 + 32 * (sl - p.bit0) + j;
      const bool lbit = v < p.n_vars && root[v].x >= 1;
      const bool ubit = v >= p.n_vars || root[v].y >= 1;
      lw |= lbit ? (1u << j) : 0u;
      uw |= ubit ? (1u << j) : 0u;
    }
    root_store[sl] = make_int2(static_cast<int>(lw), static_cast<int>(uw));
  }
  m->bit0 = p.bit0;
  m->n_slots = p.n_slots;
  if (cudaMalloc(&m->d_mem, total) != cudaSuccess) {
    (void)cudaGetLastError();
    delete m;
    return PCCP_ERR_CUDA;
  }
  m->d_root = reinterpret_cast<int2*>(m->d_mem + root_off);
  int32_t* d_iof = reinterpret_cast<int32_t*>(m->d_root + p.n_vars);
  if (cudaMemcpy(m->d_mem, p.image.data(), p.image.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_root, root.data(), root.size() * sizeof(int2), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(d_iof, iof.data(), iof.size() * sizeof(int32_t), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(d_iof + p.n_vars, uof.data(), uof.size() * sizeof(int32_t),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_root + 2 * static_cast<size_t>(p.n_vars), root_store.data(),
                 root_store.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(m->d_mem);
    delete m;
    return PCCP_ERR_CUDA;
  }
  *out = m;
  return PCCP_OK;
}

void pccp_model_destroy(pccp_model* m) {
  if (!m) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  host_pipe_free(m->pipe);
  cudaFree(m->d_mem);
  if (prev >= 0) cudaSetDevice(prev);
  delete m;
}

int pccp_model_get_info(const pccp_model* m, pccp_model_info* info) {
  if (!m || !info) return PCCP_ERR_INVALID;
  info->n_vars = m->n_vars;
  info->n_temporal = m->n_t;
  info->n_linear = m->n_lin;
  info->n_terms = m->n_terms;
  info->n_reified = m->n_rf;
  info->table_bytes = static_cast<int32_t>(m->image_bytes);
  info->bytes_per_sweep = m->bytes_per_sweep;
  const int smem_max = max_dyn_smem();
  int64_t room = static_cast<int64_t>(smem_max) - m->core_bytes - 32;
  info->max_store_vars = room > 0 ? static_cast<int32_t>(std::min<int64_t>(room / 8, 65535)) : 0;
  info->n_segments = m->n_seg;
  info->reordered = m->reordered;
  info->bool_vars = m->n_vars - m->bit0;
  info->store_bytes = 8 * m->n_slots;
  info->temporal_levels = m->n_tlev;
  return PCCP_OK;
}

int pccp_propagate_ex(const pccp_model* m, int32_t n_stores, int32_t* lb, int32_t* ub,
                      int32_t* status, int32_t* iterations, int32_t* work,
                      const pccp_launch_config* cfg, void* stream) {
  if (!m || n_stores < 0) return PCCP_ERR_INVALID;
  if (n_stores == 0) return PCCP_OK;
  if (!lb || !ub || !status) return PCCP_ERR_INVALID;
  int rc = check_device(m);
  if (rc != PCCP_OK) return rc;
  PropPlan plan;
  rc = plan_propagate(m, n_stores, cfg, &plan);
  if (rc != PCCP_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* counter = nullptr;
  PCCP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&counter), sizeof(int), s));
  PCCP_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
  rc = launch_propagate(m, plan, n_stores, lb, ub, status, iterations, work, cfg, counter, s);
  cudaFreeAsync(counter, s);
  return rc;
}

int pccp_propagate(const pccp_model* m, int32_t n_stores, int32_t* lb, int32_t* ub,
                   int32_t* status, int32_t* iterations, void* stream) {
  return pccp_propagate_ex(m, n_stores, lb, ub, status, iterations, nullptr, nullptr, stream);
}

int pccp_solve_batch(const pccp_model* const* models, int32_t n_models,
                     const pccp_solve_opts* opts, pccp_result* results, void* stream) {
  if (!models || n_models < 0 || !opts || !results) return PCCP_ERR_INVALID;
  if (n_models == 0) return PCCP_OK;
  {
    const int rc0 = check_strategy(opts);
    if (rc0 != PCCP_OK) return rc0;
  }
  if (!opts->deterministic) {  // every team over one shared queue of subproblems
    for (int32_t i = 0; i < n_models; ++i) {
      if (!models[i]) return PCCP_ERR_INVALID;
      const int rc = check_device(models[i]);
      if (rc != PCCP_OK) return rc;
    }
    return solve_queue(models, n_models, opts, results, static_cast<cudaStream_t>(stream));
  }
  std::vector<InstanceDesc> desc(n_models);
  std::vector<int32_t> woff(n_models);
  int64_t wit_total = 0;
  for (int32_t i = 0; i < n_models; ++i) {
    const pccp_model* m = models[i];
    if (!m) return PCCP_ERR_INVALID;
    const int rc = check_device(m);
    if (rc != PCCP_OK) return rc;
    woff[i] = static_cast<int32_t>(wit_total);
    wit_total += m->n_vars;
    if (wit_total > INT32_MAX) return PCCP_ERR_INVALID;
  }
  BatchPlan plan;
  {
    const int rc = plan_batch(models, n_models, opts, false, &plan);
    if (rc != PCCP_OK) return rc;
  }
  const std::vector<int32_t> ord = batch_order(models, n_models);
  for (int32_t q = 0; q < n_models; ++q)
    desc[q] = instance_desc(models[ord[q]], ord[q], woff[ord[q]]);
  const int n_teams = plan.grid * plan.teams;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // one scratch allocation: descriptors | results | witnesses | stacks | counter
  const size_t o_desc = 0;
  const size_t o_res = align16(o_desc + desc.size() * sizeof(InstanceDesc));
  const size_t o_wit = align16(o_res + static_cast<size_t>(n_models) * sizeof(InstanceResult));
  const size_t o_stk = align16(o_wit + static_cast<size_t>(wit_total) * sizeof(int32_t));
  // decision stacks in global memory only for the streamed one-team kernel
  // (k_solve_slots keeps each team's stack in its slot)
  const size_t stacks = plan.slots ? 0 : static_cast<size_t>(n_teams) * plan.max_depth;
  const size_t o_cnt = align16(o_stk + stacks * sizeof(int2));
  const size_t total = o_cnt + 16;
  uint8_t* dmem = nullptr;
  PCCP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&dmem), total, s));
  int rc = PCCP_OK;
  std::vector<InstanceResult> hres(n_models);
  std::vector<int32_t> hwit(static_cast<size_t>(wit_total));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  do {
    if (cudaMemcpyAsync(dmem + o_desc, desc.data(), desc.size() * sizeof(InstanceDesc),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(dmem + o_res, 0, static_cast<size_t>(n_models) * sizeof(InstanceResult),
                        s) != cudaSuccess ||
        cudaMemsetAsync(dmem + o_cnt, 0, 16, s) != cudaSuccess) {
      rc = PCCP_ERR_CUDA;
      break;
    }
    SolveArgs a = batch_args(plan, opts, n_models);
    a.inst = reinterpret_cast<const InstanceDesc*>(dmem + o_desc);
    a.res = reinterpret_cast<InstanceResult*>(dmem + o_res);
    a.witness = reinterpret_cast<int32_t*>(dmem + o_wit);
    a.stacks = reinterpret_cast<int2*>(dmem + o_stk);
    a.counter = reinterpret_cast<int*>(dmem + o_cnt);
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = PCCP_ERR_CUDA;
      break;
    }
    cudaEventRecord(e0, s);
    plan.kern<<<plan.grid, plan.team * plan.teams, plan.smem, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) {
      rc = PCCP_ERR_CUDA;
      break;
    }
    cudaEventRecord(e1, s);
    if (cudaMemcpyAsync(hres.data(), dmem + o_res,
                        static_cast<size_t>(n_models) * sizeof(InstanceResult),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hwit.data(), dmem + o_wit, hwit.size() * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = PCCP_ERR_CUDA;
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(dmem, s);
  if (rc != PCCP_OK) {
    (void)cudaGetLastError();
    return rc;
  }
  for (int32_t i = 0; i < n_models; ++i) {
    const InstanceResult& r = hres[i];
    pccp_result& o = results[i];
    o.status = r.status;
    o.has_solution = r.has_solution;
    o.objective = r.objective;
    o.nodes = r.nodes;
    o.fails = r.fails;
    o.solutions = r.solutions;
    o.iterations = r.iterations;
    const pccp_model* m = models[i];
    o.rows_evaluated = r.evals;
    o.max_depth = r.max_depth;
    o.elapsed_ms = ms;
    o.model_ms = r.us / 1000.f;
    if (o.witness && r.has_solution)
      std::memcpy(o.witness, hwit.data() + woff[i],
                  static_cast<size_t>(m->n_vars) * sizeof(int32_t));
    if (r.error == 1 || r.error == 3) rc = PCCP_ERR_TIMEOUT;
    if (r.error == 2) rc = PCCP_ERR_INVALID;
  }
  return rc;
}

}  // extern "C"

namespace {

// The EPS kernel pair for a search's options.
template <bool kGlobal, bool kStream>
void eps_kernels(bool learned, bool skip_stable, void (**kexp)(EpsArgs),
                 void (**ksol)(EpsArgs)) {
  *kexp = learned ? k_eps_expand<false, true, kGlobal, kStream>
                  : (skip_stable ? k_eps_expand<true, false, kGlobal, kStream>
                                 : k_eps_expand<false, false, kGlobal, kStream>);
  *ksol = learned ? k_eps_solve<false, true, kGlobal, kStream>
                  : (skip_stable ? k_eps_solve<true, false, kGlobal, kStream>
                                 : k_eps_solve<false, false, kGlobal, kStream>);
}

// Parallel search of one model: breadth-first frontier growth, then one
// persistent launch over the frontier's subproblems (k_solve_eps.cuh).
int solve_parallel(const pccp_model* m, const pccp_solve_opts* o, pccp_result* res,
                   cudaStream_t s) {
  const int smem_max = max_dyn_smem();
  const int sms = sm_count();
  if (smem_max <= 0 || sms <= 0) return PCCP_ERR_CUDA;
  int team = o->threads > 0 ? o->threads : 128;
  if (team % 32 != 0 || team > 1024) return PCCP_ERR_INVALID;
  const int xw = policy_x_words(o, m->n_branch);
  const size_t per_team = sizeof(EpsCtrl) + 4 * ((track_words(m->n_vars, m->n_lin) + 3) & ~3) +
                          static_cast<size_t>(m->n_slots) * sizeof(int2) +
                          4 * static_cast<size_t>(xw);
  const uint32_t img_smem =
      (o->strategy != PCCP_LEARNED && use_skip_stable(o->skip_stable, false)) ? m->track_bytes
                                                                              : m->core_bytes;
  const bool global = m->bit0 < m->n_vars || static_cast<size_t>(img_smem) + 16 + per_team >
                                                  static_cast<size_t>(smem_max);
  const size_t base = (global ? 0 : static_cast<size_t>(img_smem)) + 16;
  if (base + per_team > static_cast<size_t>(smem_max)) return PCCP_ERR_SMEM;
  if (global && o->threads <= 0) team = 1024;
  const int fit = static_cast<int>((static_cast<size_t>(smem_max) - base) / per_team);
  const int teams = std::max(1, std::min({8, fit, 1024 / team}));
  const int stages =
      global ? stream_stages_for(m->n_seg, o->stream_table, base, per_team, teams, smem_max) : 0;
  const size_t smem = base + static_cast<size_t>(teams) * (per_team + stream_bytes(stages));
  const bool learned = o->strategy == PCCP_LEARNED;
  using EpsKernel = void (*)(EpsArgs);
  EpsKernel kexp, ksol;
  if (stages > 0)
    eps_kernels<true, true>(learned, use_skip_stable(o->skip_stable, true), &kexp, &ksol);
  else if (global)
    eps_kernels<true, false>(learned, use_skip_stable(o->skip_stable, true), &kexp, &ksol);
  else
    eps_kernels<false, false>(learned, use_skip_stable(o->skip_stable, false), &kexp, &ksol);
  PCCP_CUDA(allow_smem(reinterpret_cast<const void*>(kexp), smem));
  PCCP_CUDA(allow_smem(reinterpret_cast<const void*>(ksol), smem));
  int occ_e = 0, occ_s = 0;
  PCCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_e, kexp, teams * team, smem));
  PCCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, ksol, teams * team, smem));
  const int per_sm = std::min(occ_e, occ_s);
  if (per_sm < 1) return PCCP_ERR_SMEM;
  int grid = sms * per_sm;
  if (o->blocks > 0) grid = std::min(grid, static_cast<int>(o->blocks));
  const int n_teams = grid * teams;
  const int max_depth = m->max_decisions;
  const int target = 4 * n_teams;
  constexpr int kMaxSeedLen = 48;
  const size_t cap = 2 * static_cast<size_t>(target);
  const size_t level_bytes = cap * (kMaxSeedLen + 1) * sizeof(int2);

  const size_t o_g = 0;
  const size_t o_tb = align16(o_g + sizeof(EpsGlobal));
  const size_t o_th = align16(o_tb + static_cast<size_t>(n_teams) * sizeof(int));
  const size_t o_w = align16(o_th + static_cast<size_t>(n_teams) * sizeof(int));
  const size_t o_stk = align16(o_w + static_cast<size_t>(n_teams) * m->n_vars * sizeof(int32_t));
  const size_t o_la = align16(o_stk + static_cast<size_t>(n_teams) * max_depth * sizeof(int2));
  const size_t o_lb = align16(o_la + level_bytes);
  const size_t o_cnt = align16(o_lb + level_bytes);
  const size_t total = o_cnt + 16;
  uint8_t* d = nullptr;
  PCCP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), total, s));
  int rc = PCCP_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  EpsGlobal hg;
  std::vector<int> tbest(n_teams), thas(n_teams);
  int n_final = 0, final_len = 0;
  uint8_t* final_paths = nullptr;
  do {
    std::memset(&hg, 0, sizeof(hg));
    hg.best = INT_MAX;
    if (cudaMemsetAsync(d, 0, o_la, s) != cudaSuccess ||
        cudaMemcpyAsync(d + o_g, &hg, sizeof(hg), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = PCCP_ERR_CUDA;
      break;
    }
    EpsArgs a;
    std::memset(&a, 0, sizeof(a));
    a.image = m->d_mem;
    a.root = m->d_root;
    a.image_bytes = global ? m->image_bytes : img_smem;
    a.g = reinterpret_cast<EpsGlobal*>(d + o_g);
    a.team_best = reinterpret_cast<int*>(d + o_tb);
    a.team_has = reinterpret_cast<int*>(d + o_th);
    a.witness = reinterpret_cast<int32_t*>(d + o_w);
    a.stacks = reinterpret_cast<int2*>(d + o_stk);
    a.in_counter = reinterpret_cast<int*>(d + o_cnt);
    a.out_count = reinterpret_cast<int*>(d + o_cnt + 4);
    a.n_vars = m->n_vars;
    a.n_slots = m->n_slots;
    a.max_iter = m->max_iter;
    a.teams = teams;
    a.team_size = team;
    a.max_depth = max_depth;
    a.mode = o->mode;
    a.strategy = o->strategy;
    a.obj_ub = o->obj_ub;
    a.levels = levels_mask(o->temporal_levels, false);
    a.track_words = track_words(m->n_vars, m->n_lin);
    a.table_global = global ? 1 : 0;
    a.stream_stages = stages;
    a.x_words = xw;
    a.policy = o->strategy == PCCP_LEARNED ? policy_dev(o->policy) : nullptr;
    a.node_limit = o->node_limit;
    a.time_limit_ns = o->time_limit_ms > 0 ? o->time_limit_ms * 1000000ll : 0;
    uint8_t* lin = d + o_la;
    uint8_t* lout = d + o_lb;
    int n_in = 1, len = 0;
    bool finished = false;
    cudaEventRecord(e0, s);
    // breadth-first growth of the frontier
    while (n_in < target && len < kMaxSeedLen) {
      a.in_paths = reinterpret_cast<const int2*>(lin);
      a.out_paths = reinterpret_cast<int2*>(lout);
      a.n_in = n_in;
      a.in_len = len;
      a.out_cap = static_cast<int>(cap);
      if (cudaMemsetAsync(d + o_cnt, 0, 16, s) != cudaSuccess) {
        rc = PCCP_ERR_CUDA;
        break;
      }
      kexp<<<grid, teams * team, smem, s>>>(a);
      if (cudaGetLastError() != cudaSuccess) {
        rc = PCCP_ERR_CUDA;
        break;
      }
      int n_out = 0;
      if (cudaMemcpyAsync(&n_out, a.out_count, sizeof(int), cudaMemcpyDeviceToHost, s) !=
              cudaSuccess ||
          cudaMemcpyAsync(&hg, d + o_g, sizeof(hg), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        rc = PCCP_ERR_CUDA;
        break;
      }
      if (hg.error || hg.stop || n_out == 0) {
        finished = true;  // error, limit, satisfied, or the tree ended while growing
        break;
      }
      std::swap(lin, lout);
      n_in = n_out;
      ++len;
    }
    if (rc != PCCP_OK) break;
    if (!finished) {
      n_final = n_in;
      final_len = len;
      final_paths = lin;
      a.in_paths = reinterpret_cast<const int2*>(final_paths);
      a.out_paths = nullptr;
      a.n_in = n_final;
      a.in_len = final_len;
      a.out_cap = 0;
      if (cudaMemsetAsync(d + o_cnt, 0, 16, s) != cudaSuccess) {
        rc = PCCP_ERR_CUDA;
        break;
      }
      ksol<<<grid, teams * team, smem, s>>>(a);
      if (cudaGetLastError() != cudaSuccess) {
        rc = PCCP_ERR_CUDA;
        break;
      }
    }
    cudaEventRecord(e1, s);
    if (cudaMemcpyAsync(&hg, d + o_g, sizeof(hg), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(tbest.data(), d + o_tb, n_teams * sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(thas.data(), d + o_th, n_teams * sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = PCCP_ERR_CUDA;
      break;
    }
    int winner = -1;
    for (int t = 0; t < n_teams; ++t) {
      if (!thas[t]) continue;
      if (o->mode == PCCP_OPTIMISE && m->objective >= 0 && tbest[t] != hg.best) continue;
      winner = t;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    res->has_solution = winner >= 0;
    res->objective = winner >= 0 ? tbest[winner] : 0;
    res->nodes = static_cast<int64_t>(hg.nodes);
    res->fails = static_cast<int64_t>(hg.fails);
    res->solutions = static_cast<int64_t>(hg.solutions);
    res->iterations = static_cast<int64_t>(hg.iterations);
    res->rows_evaluated = static_cast<int64_t>(hg.evals);
    res->max_depth = hg.max_depth;
    res->elapsed_ms = ms;
    res->model_ms = 0.f;
    res->status = hg.limited ? PCCP_RES_LIMIT
                             : (res->has_solution ? PCCP_RES_OPTIMAL : PCCP_RES_INFEASIBLE);
    if (res->witness && winner >= 0) {
      if (cudaMemcpyAsync(res->witness, d + o_w + static_cast<size_t>(winner) * m->n_vars * 4,
                          static_cast<size_t>(m->n_vars) * sizeof(int32_t), cudaMemcpyDeviceToHost,
                          s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        rc = PCCP_ERR_CUDA;
        break;
      }
    }
    if (hg.error == 1 || hg.error == 3) rc = PCCP_ERR_TIMEOUT;
    if (hg.error == 2 || hg.error == 4) rc = PCCP_ERR_INVALID;
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(d, s);
  if (rc != PCCP_OK) (void)cudaGetLastError();
  return rc;
}

}  // namespace

namespace {

// Launch plan of the parallel search over the shared queue.
struct QueuePlan {
  void (*kern)(QArgs);
  int team, teams, grid, max_len, xw;
  int mode;  // queue_kernel's mode
  size_t smem;
  uint32_t slot_bytes, off_track, off_x, off_stack, off_store;
  bool shared, table_global;
  uint32_t shared_bytes, shared_region;
};

template <int kMode>
void (*queue_kernel_t(const pccp_solve_opts* o))(QArgs) {
  if (o->strategy == PCCP_LEARNED) return k_search_queue<false, false, true, kMode>;
  if (o->skip_stable > 0) return k_search_queue<true, true, false, kMode>;
  if (o->skip_stable < 0) return k_search_queue<false, false, false, kMode>;
  return k_search_queue<false, true, false, kMode>;
}
// mode 0: a slot per team (many models); 1: one model, table shared in the
// CTA; 2: one model, table read in place; 3: mode 2 with Booleans as bits
void (*queue_kernel(const pccp_solve_opts* o, int mode))(QArgs) {
  return mode == 0   ? queue_kernel_t<0>(o)
         : mode == 1 ? queue_kernel_t<1>(o)
         : mode == 2 ? queue_kernel_t<2>(o)
                     : queue_kernel_t<3>(o);
}

// Team size of a search when the caller leaves it to the library: enough
// threads for about two rows each of the largest model, in whole warps, at
// least 64 and at most `cap` (small models: small teams, so more of them).
int default_team(int max_rows, int cap) {
  return std::min(cap, std::max(64, ((max_rows + 1) / 2 + 31) & ~31));
}

int plan_queue(const pccp_model* const* models, int32_t n, const pccp_solve_opts* o,
               QueuePlan* p, bool any_strategy = false) {
  const int smem_max = max_dyn_smem();
  const int sms = sm_count();
  if (smem_max <= 0 || sms <= 0) return PCCP_ERR_CUDA;
  if (o->threads < 0 || o->threads % 32 != 0 || o->threads > 1024) return PCCP_ERR_INVALID;
  if (o->teams_per_cta < 0 || o->teams_per_cta > kMaxTeamsPerCta) return PCCP_ERR_INVALID;
  int32_t max_vars = 0, max_branch = 0, max_tw = 0, max_rows = 0, max_dec = 2;
  for (int32_t i = 0; i < n; ++i) {
    const pccp_model* m = models[i];
    max_vars = std::max(max_vars, m->n_vars);
    max_branch = std::max(max_branch, m->n_branch);
    max_tw = std::max(max_tw, track_words(m->n_vars, m->n_lin));
    max_rows = std::max(max_rows, m->n_t + m->n_rf + m->n_lin);
    max_dec = std::max(max_dec, m->max_decisions);
  }
  p->xw = any_strategy ? 24 * ((max_branch + 15) & ~15) : policy_x_words(o, max_branch);
  p->max_len = max_dec;
  p->off_track = static_cast<uint32_t>(align16(16 + sizeof(QCtrl)));
  p->off_x = p->off_track + 4u * static_cast<uint32_t>((max_tw + 3) & ~3);
  p->off_stack = static_cast<uint32_t>(align16(p->off_x + 4u * static_cast<uint32_t>(p->xw)));
  p->off_store = static_cast<uint32_t>(
      align16(p->off_stack + sizeof(int2) * static_cast<size_t>(p->max_len)));
  const bool learned = o->strategy == PCCP_LEARNED;
  const bool track_s = !learned && o->skip_stable > 0;
  p->shared = n == 1;
  if (p->shared) {
    // one model: its table once per CTA, shared by the CTA's teams
    const pccp_model* m = models[0];
    uint32_t per = static_cast<uint32_t>(
        (p->off_store + 8ull * static_cast<uint32_t>(m->n_slots) + 127u) & ~127ull);
    const uint32_t img = track_s ? m->track_bytes : m->core_bytes;
    const uint32_t region = ((img + 127u) & ~127u) + 128u;
    p->table_global = m->bit0 < m->n_vars ||  // bit layouts are read in place
                      static_cast<size_t>(region) + per > static_cast<size_t>(smem_max);
    if (per > static_cast<uint32_t>(smem_max)) return PCCP_ERR_SMEM;
    if (p->table_global) {  // room for the temporal levels after each team's store
      const uint32_t with =
          (slot_need_global(m, p->off_store, static_cast<uint32_t>(smem_max)) + 127u) & ~127u;
      if (static_cast<size_t>(with) * std::max(1, static_cast<int>(o->teams_per_cta)) <=
          static_cast<size_t>(smem_max))
        per = with;
    }
    p->shared_bytes = p->table_global ? 0u : img;
    p->shared_region = p->table_global ? 0u : region;
    int team = o->threads;
    if (team == 0 && o->props_per_thread > 0)
      team = std::min(1024, std::max(32, ((max_rows + o->props_per_thread - 1) /
                                              o->props_per_thread + 31) & ~31));
    if (team == 0) team = p->table_global ? 1024 : default_team(max_rows, 128);
    const int fit = static_cast<int>((static_cast<uint32_t>(smem_max) - p->shared_region) / per);
    int teams = o->teams_per_cta > 0 ? o->teams_per_cta : 8;
    teams = std::min({teams, fit, 1024 / team});
    if (teams < 1 || (o->teams_per_cta > 0 && teams < o->teams_per_cta)) return PCCP_ERR_SMEM;
    p->team = team;
    p->teams = teams;
    p->slot_bytes = per;
    p->smem = p->shared_region + static_cast<size_t>(teams) * per;
    p->mode = !p->table_global ? 1 : models[0]->bit0 < models[0]->n_vars ? 3 : 2;
    p->kern = queue_kernel(o, p->mode);
  } else {
    // many models: a slot per team, as the batched search plans them
    pccp_solve_opts q = *o;
    if (q.threads == 0 && q.props_per_thread == 0) q.threads = default_team(max_rows, 256);
    BatchPlan bp;
    const int rc = plan_batch(models, n, &q, false, &bp);
    if (rc != PCCP_OK) return rc;
    if (!bp.slots) return PCCP_ERR_INVALID;  // streaming is not offered here
    // the same choices with this kernel's control block
    const int teams = bp.teams;
    const uint32_t room = static_cast<uint32_t>(smem_max / teams) & ~127u;
    uint32_t want = 0;
    for (int32_t i = 0; i < n; ++i) {
      const uint32_t staged = slot_need(models[i], p->off_store, track_s, true);
      want = std::max(want, staged <= room ? staged
                                           : slot_need_global(models[i], p->off_store, room));
    }
    if (want > room) return PCCP_ERR_SMEM;
    p->shared_bytes = p->shared_region = 0;
    p->table_global = false;
    p->team = bp.team;
    p->teams = teams;
    p->slot_bytes = (want + 127u) & ~127u;
    p->smem = static_cast<size_t>(teams) * p->slot_bytes;
    p->mode = 0;
    p->kern = queue_kernel(o, 0);
  }
  void (*kerns[8])(QArgs) = {p->kern};
  int n_kerns = 1;
  if (any_strategy) {  // a batch planned once for every later search
    pccp_solve_opts q = *o;
    const int mode = p->mode;
    for (int strategy : {PCCP_INPUT_ORDER, PCCP_LEARNED})
      for (int skip : {-1, 0, 1}) {
        q.strategy = strategy;
        q.skip_stable = skip;
        if (n_kerns < 8) kerns[n_kerns++] = queue_kernel(&q, mode);
      }
  }
  int per_sm = 1 << 30;
  for (int ki = 0; ki < n_kerns; ++ki) {
    PCCP_CUDA(allow_smem(reinterpret_cast<const void*>(kerns[ki]), p->smem));
    int occ = 0;
    PCCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kerns[ki], p->team * p->teams,
                                                            p->smem));
    per_sm = std::min(per_sm, occ);
  }
  if (per_sm < 1) return PCCP_ERR_SMEM;
  p->grid = sms * per_sm;
  if (o->blocks > 0) p->grid = std::min(p->grid, static_cast<int>(o->blocks));
  return PCCP_OK;
}

// Ring capacity of a queue search: every root, then room for donations.
size_t queue_cap(int32_t n, int n_teams, int max_len) {
  const size_t per_item = static_cast<size_t>(max_len) * sizeof(int2);
  return std::max<size_t>(static_cast<size_t>(n) + 2 * static_cast<size_t>(n_teams),
                          std::min<size_t>(65536, (96u << 20) / per_item));
}

// Option-dependent kernel arguments of a queue search.
void queue_opts_args(const pccp_solve_opts* o, QArgs* a) {
  a->policy = o->strategy == PCCP_LEARNED ? policy_dev(o->policy) : nullptr;
  a->mode = o->mode;
  a->strategy = o->strategy;
  a->obj_ub = o->obj_ub;
  a->levels = levels_mask(o->temporal_levels, false);
  a->donate_nodes = o->donate_nodes < 0 ? -1 : (o->donate_nodes > 0 ? o->donate_nodes : 4);
  a->granularity = o->queue_granularity > 0 ? o->queue_granularity : 1;
  a->node_limit = o->node_limit;
  a->time_limit_ns = o->time_limit_ms > 0 ? o->time_limit_ms * 1000000ll : 0;
}

// Results of a queue search from the per-model states.
int queue_results(const pccp_model* const* models, int32_t n, const QModel* hq,
                  const QGlobal& hg, const int32_t* hwit, const int32_t* woff, float ms,
                  pccp_result* results) {
  for (int32_t i = 0; i < n; ++i) {
    const QModel& q = hq[i];
    pccp_result& r = results[i];
    const bool has = q.has != 0;
    r.has_solution = has;
    r.objective = has ? q.wit_obj : 0;
    // complete: satisfied, or every item of the model exhausted untouched by
    // a limit (items left in the queue by a stop keep outstanding above 0)
    if (q.done == 1 || (q.outstanding == 0 && !q.cut && hg.error == 0))
      r.status = has ? PCCP_RES_OPTIMAL : PCCP_RES_INFEASIBLE;
    else
      r.status = PCCP_RES_LIMIT;
    r.nodes = static_cast<int64_t>(q.nodes);
    r.fails = static_cast<int64_t>(q.fails);
    r.solutions = static_cast<int64_t>(q.sols);
    r.iterations = static_cast<int64_t>(q.iters);
    r.rows_evaluated = static_cast<int64_t>(q.evals);
    r.max_depth = q.max_depth;
    r.elapsed_ms = ms;
    r.model_ms = q.outstanding == 0 ? static_cast<float>(q.t_done) * 1e-6f : 0.f;
    if (r.witness && has && hwit)
      std::memcpy(r.witness, hwit + woff[i],
                  static_cast<size_t>(models[i]->n_vars) * sizeof(int32_t));
  }
  if (hg.error == 1 || hg.error == 3 || hg.error == 4) return PCCP_ERR_TIMEOUT;
  if (hg.error == 2) return PCCP_ERR_INVALID;
  return PCCP_OK;
}

// Plan-dependent kernel arguments of a queue search.
void queue_plan_args(const QueuePlan& plan, int32_t n, size_t cap, QArgs* a) {
  a->n_models = n;
  a->cap = static_cast<int>(cap);
  a->max_len = plan.max_len;
  a->n_teams = plan.grid * plan.teams;
  a->team_size = plan.team;
  a->teams = plan.teams;
  a->slot_bytes = plan.slot_bytes;
  a->off_track = plan.off_track;
  a->off_x = plan.off_x;
  a->off_stack = plan.off_stack;
  a->off_store = plan.off_store;
  a->shared_table = plan.shared ? 1 : 0;
  a->table_global = plan.table_global ? 1 : 0;
  a->shared_bytes = plan.shared_bytes;
  a->shared_region = plan.shared_region;
}

// Parallel search of n models over one shared queue (see k_search_queue.inc).
int solve_queue(const pccp_model* const* models, int32_t n, const pccp_solve_opts* o,
                pccp_result* results, cudaStream_t s) {
  QueuePlan plan;
  int rc = plan_queue(models, n, o, &plan);
  if (rc != PCCP_OK) return rc;
  const int n_teams = plan.grid * plan.teams;
  std::vector<InstanceDesc> desc(n);
  std::vector<int32_t> woff(n);
  int64_t wit_total = 0;
  for (int32_t i = 0; i < n; ++i) {
    woff[i] = static_cast<int32_t>(wit_total);
    wit_total += models[i]->n_vars;
    if (wit_total > INT32_MAX) return PCCP_ERR_INVALID;
    desc[i] = instance_desc(models[i], i, woff[i]);
  }
  const size_t per_item = static_cast<size_t>(plan.max_len) * sizeof(int2);
  const size_t cap = queue_cap(n, n_teams, plan.max_len);
  if (cap > static_cast<size_t>(INT32_MAX)) return PCCP_ERR_INVALID;
  const size_t o_g = 0;
  const size_t o_qm = align16(o_g + sizeof(QGlobal));
  const size_t o_desc = align16(o_qm + static_cast<size_t>(n) * sizeof(QModel));
  const size_t o_seq = align16(o_desc + static_cast<size_t>(n) * sizeof(InstanceDesc));
  const size_t o_hdr = align16(o_seq + cap * sizeof(unsigned long long));
  const size_t o_path = align16(o_hdr + cap * sizeof(int2));
  const size_t o_wit = align16(o_path + cap * per_item);
  const size_t total = align16(o_wit + static_cast<size_t>(wit_total) * sizeof(int32_t));
  uint8_t* d = nullptr;
  PCCP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), total, s));
  QArgs a;
  std::memset(&a, 0, sizeof(a));
  a.inst = reinterpret_cast<const InstanceDesc*>(d + o_desc);
  a.qm = reinterpret_cast<QModel*>(d + o_qm);
  a.g = reinterpret_cast<QGlobal*>(d + o_g);
  a.seq = reinterpret_cast<unsigned long long*>(d + o_seq);
  a.hdr = reinterpret_cast<int2*>(d + o_hdr);
  a.path = reinterpret_cast<int2*>(d + o_path);
  a.witness = reinterpret_cast<int32_t*>(d + o_wit);
  queue_plan_args(plan, n, cap, &a);
  queue_opts_args(o, &a);
  std::vector<QModel> hq(n);
  QGlobal hg;
  std::vector<int32_t> hwit(static_cast<size_t>(wit_total));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  rc = PCCP_OK;
  do {
    if (cudaMemcpyAsync(d + o_desc, desc.data(), desc.size() * sizeof(InstanceDesc),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = PCCP_ERR_CUDA;
      break;
    }
    k_queue_init<<<256, 256, 0, s>>>(a);
    cudaEventRecord(e0, s);
    plan.kern<<<plan.grid, plan.team * plan.teams, plan.smem, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) {
      rc = PCCP_ERR_CUDA;
      break;
    }
    cudaEventRecord(e1, s);
    if (cudaMemcpyAsync(hq.data(), d + o_qm, hq.size() * sizeof(QModel), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaMemcpyAsync(&hg, d + o_g, sizeof(hg), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hwit.data(), d + o_wit, hwit.size() * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = PCCP_ERR_CUDA;
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(d, s);
  if (rc != PCCP_OK) {
    (void)cudaGetLastError();
    return rc;
  }
  return queue_results(models, n, hq.data(), hg, hwit.data(), woff.data(), ms, results);
}

}  // namespace

extern "C" {

int pccp_solve(const pccp_model* m, const pccp_solve_opts* opts, pccp_result* result,
               void* stream) {
  if (!m || !opts || !result) return PCCP_ERR_INVALID;
  {
    const int rc0 = check_strategy(opts);
    if (rc0 != PCCP_OK) return rc0;
  }
  if (!opts->deterministic) {
    const int rc = check_device(m);
    if (rc != PCCP_OK) return rc;
    // streamed tables keep the frontier-then-persistent search
    // (k_eps_expand / k_eps_solve); otherwise the shared queue with donation
    if (opts->stream_table > 0) {
      const int smem_max = max_dyn_smem();
      if (smem_max <= 0) return PCCP_ERR_CUDA;
      if (static_cast<int64_t>(m->core_bytes) + 128 + 8ll * m->n_vars + 4096 > smem_max)
        return solve_parallel(m, opts, result, static_cast<cudaStream_t>(stream));
    }
    const pccp_model* one[1] = {m};
    return solve_queue(one, 1, opts, result, static_cast<cudaStream_t>(stream));
  }
  pccp_solve_opts o = *opts;
  if (o.threads <= 0) o.threads = 512;
  o.teams_per_cta = 1;  // one model: one team
  const pccp_model* one[1] = {m};
  return pccp_solve_batch(one, 1, &o, result, stream);
}

}  // extern "C"

#include "pccp_noalloc.inc"
#include "pccp_batch.inc"
#include "pccp_policy.inc"
#include "pccp_host.inc"
