// k_solve_eps.cuh -- parallel search of one model by every team of the GPU
// (included by pccp.cu).
//
// Embarrassingly parallel search (the EPS variant of Sec. 5): the tree is
// first grown breadth first, one level per launch of k_eps_expand, until the
// frontier holds enough subproblems for every team; each subproblem is a
// decision path.  k_eps_solve then runs persistent teams that pull paths from
// a global counter and search each subtree depth first with full
// recomputation from the root store (Sec. 5).  The teams share the incumbent
// through a global atomicMin: every node is told ub(obj) <= best - 1 with the
// best objective known when the node starts (branch and bound).
#pragma once

#include "pccp_device.cuh"
#include "policy.cuh"

namespace pccp {

// Search state shared by every team of both kernels (global memory).
struct EpsGlobal {
  int best;      // incumbent objective, INT_MAX while none
  int stop;      // 1: stop at the next node (limit reached, or satisfied)
  int limited;   // a node or time limit stopped the search
  int error;     // 1 iteration budget, 2 decision stack, 3 table load, 4 frontier overflow
  unsigned long long t0;          // globaltimer at the first node (0 until set)
  unsigned long long live_nodes;  // node count published in batches, for the limit
  unsigned long long nodes, fails, solutions, iterations, evals;
  int max_depth;
  int pad[3];
};

struct EpsArgs {
  const uint8_t* image;
  const int2* root;
  EpsGlobal* g;
  int* team_best;        // [n_teams]: objective of the team's recorded witness
  int* team_has;         // [n_teams]: 1 if the team recorded a witness
  int32_t* witness;      // [n_teams][n_vars]
  int2* stacks;          // [n_teams][max_depth]
  const int2* in_paths;  // [n_in][in_len]
  int2* out_paths;       // [out_cap][in_len + 1] (expansion only)
  int* in_counter;
  int* out_count;
  uint32_t image_bytes;
  int n_vars;
  int n_slots;           // store slots (variables below bit0, then Boolean words)
  int max_iter;
  int teams;             // per CTA
  int team_size;
  int n_in;
  int in_len;
  int out_cap;
  int max_depth;
  int mode;
  int strategy;
  int obj_ub;
  int track_words;
  int table_global;  // 1: rows are read from the device image
  int stream_stages; // table_global: buffers of each team's stream (0: rows read in place)
  int x_words;       // learned strategy: feature rows per team (words)
  const PolicyDev* policy;
  int64_t node_limit;
  int64_t time_limit_ns;
  int levels;  // temporal levels: bit 0 staged tables, bit 1 global ones
};

struct EpsCtrl {
  unsigned long long sel[2];
  FixCtrl fc;
  int stop;
  int record;
  int err;
  int depth;
  int next;
  int out;
  int cur_depth;  // P1: depth of the node (features of the learned strategy)
  int pad;
};

enum : int { kNodeFailed = 0, kNodeSolution = 1, kNodeBranch = 2, kNodeStop = 3, kNodeError = 4 };

__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t eps_now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One node: limits and incumbent bound (thread 0), fixed point, selection.
// The caller has put root join decisions into st; the first barrier here
// orders those writes before the fixed point.  On kNodeBranch, *key holds
// the selection key (branch index in the low 32 bits).  Team-uniform result.
// Broadcast slots follow the protocol of team_dfs: written before a barrier,
// read after it, not rewritten before another barrier has passed.
template <bool kTrack, bool kLearned, bool kGlobal, bool kStream>
__device__ __forceinline__ int eps_node(const Tab& tb, int2* st, const Team& tm, EpsCtrl* sc,
                                        const Track& tk, bool seeded, unsigned par,
                                        const EpsArgs& a, int& it, unsigned long long& key,
                                        int depth, uint32_t* X, Streamer* stream) {
  EpsGlobal* g = a.g;
  if (tm.tid == 0) {
    int stop = ld_relaxed_gpu(&g->stop);
    if (!stop && a.time_limit_ns > 0) {
      const unsigned long long t0 = *reinterpret_cast<volatile unsigned long long*>(&g->t0);
      if (t0 != 0 && static_cast<int64_t>(eps_now_ns() - t0) > a.time_limit_ns) {
        atomicExch(&g->limited, 1);
        atomicExch(&g->stop, 1);
        stop = 1;
      }
    }
    if (!stop && tb.objective >= 0) {
      int bound = a.obj_ub;
      if (a.mode == PCCP_OPTIMISE) {
        const int gb = ld_relaxed_gpu(&g->best);
        if (gb != INT_MAX) bound = min(bound, gb - 1);
      }
      if (bound < INT_MAX) {
        const int old = atom_min_s32(&st[tb.objective].y, bound);
        if (kTrack && old > bound) mark_changed(tb, tk, 2, tb.objective);
      }
    }
    sc->stop = stop;
    sc->fc.fail = 0;
    sc->fc.evals = 0;
    sc->fc.bytes = 0;
    sc->sel[par] = ~0ull;
    sc->cur_depth = depth;
  }
  team_bar(tm.bar, tm.nthr);
  if (sc->stop) return kNodeStop;
  const int fst =
      team_fixpoint<kTrack, kGlobal, kStream>(tb, st, tm, &sc->fc, tk, !seeded, a.max_iter, it,
                                              stream);
  if (fst == kError) return kNodeError;
  if (fst == kFailed) return kNodeFailed;
  unsigned long long* sel = &sc->sel[par];
  if (kLearned) {
    learned_select(tb, st, a.root, tm, a.policy, X, sel, sc->cur_depth);
  } else {
    for (int k = tm.tid; k < tb.n_branch; k += tm.nthr) {
      const int v = tb.branch[k];
      const int2 D = ld_dom(st, v);
      if (D.x < D.y) {
        unsigned long long kk = static_cast<unsigned long long>(k);
        if (a.strategy == PCCP_FIRST_FAIL)
          kk |= static_cast<unsigned long long>(static_cast<uint32_t>(D.y - D.x)) << 32;
        atomicMin(sel, kk);
        if (a.strategy == PCCP_INPUT_ORDER) break;
      }
    }
  }
  if (kTrack) track_clear02(tk, tm);  // for a left child's seeded fixed point
  team_bar(tm.bar, tm.nthr);
  key = *sel;
  return key == ~0ull ? kNodeSolution : kNodeBranch;
}

// A solution was found on st: publish it to the incumbent, record the
// team's witness when it improves (optimise) or is the team's first
// (count-all), stop everything when there is no objective.  Ends with a
// barrier; team-uniform.
__device__ __forceinline__ void eps_solution(const Tab& tb, int2* st, const Team& tm, EpsCtrl* sc,
                                             const EpsArgs& a, int team_gid,
                                             unsigned long long& sols) {
  EpsGlobal* g = a.g;
  if (tm.tid == 0) {
    ++sols;
    const int z = tb.objective >= 0 ? st[tb.objective].x : 0;
    bool record;
    if (a.mode == PCCP_OPTIMISE && tb.objective >= 0) {
      const int old = atomicMin(&g->best, z);
      record = z < old;
    } else {
      record = a.team_has[team_gid] == 0;
      if (tb.objective >= 0) atomicMin(&g->best, z);
    }
    if (a.mode == PCCP_OPTIMISE && tb.objective < 0) atomicExch(&g->stop, 1);
    if (record) {
      a.team_best[team_gid] = z;
      a.team_has[team_gid] = 1;
    }
    sc->record = record;
  }
  team_bar(tm.bar, tm.nthr);
  if (sc->record) {
    // in the caller's variable order (internal_of after the root)
    int32_t* w = a.witness + static_cast<size_t>(team_gid) * a.n_vars;
    const int32_t* internal_of = reinterpret_cast<const int32_t*>(a.root + a.n_vars);
    for (int x = tm.tid; x < a.n_vars; x += tm.nthr)
      w[x] = var_dom_plain(st, tb.bit0, __ldg(internal_of + x)).x;
  }
}

template <bool kTrack>
__device__ __forceinline__ void eps_restore(const int2* root, int2* st, const Team& tm, int nv,
                                            int n_slots, const Track& tk, const int2* path,
                                            int len) {
  // the root in the store layout follows the root box and the two index maps
  const int2* root_store = root + 2 * static_cast<size_t>(nv);
  for (int v = tm.tid; v < n_slots; v += tm.nthr) st[v] = __ldg(root_store + v);
  if (kTrack) track_clear02(tk, tm);
  team_bar(tm.bar, tm.nthr);
  for (int k = tm.tid; k < len; k += tm.nthr) {
    const int2 e = path[k];
    const int v = static_cast<int>(static_cast<uint32_t>(e.x) & 0x7fffffffu);
    if (static_cast<uint32_t>(e.x) & 0x80000000u)
      atom_max_s32(&st[v].x, e.y);
    else
      atom_min_s32(&st[v].y, e.y);
  }
}

__device__ __forceinline__ void eps_count_node(const EpsArgs& a, unsigned long long& local,
                                               unsigned long long& published) {
  ++local;
  if (a.node_limit > 0 && local - published >= 64) {
    const unsigned long long n = atomicAdd(&a.g->live_nodes, local - published) + (local - published);
    published = local;
    if (n >= static_cast<unsigned long long>(a.node_limit)) {
      atomicExch(&a.g->limited, 1);
      atomicExch(&a.g->stop, 1);
    }
  }
}

struct EpsSmem {
  uint8_t* img;
  uint64_t* mbar;
  EpsCtrl* sc;
  uint32_t* track;
  int2* st;
  uint32_t* X;       // learned strategy's feature rows
  uint8_t* stream;   // the team's stream region (streamed tables)
};

// [table image | streams: one stream region per team | none][mbarrier 16 B]
// [EpsCtrl x teams][change words x teams][stores x teams][feature rows x teams]
__device__ __forceinline__ EpsSmem eps_smem(uint8_t* smem, const EpsArgs& a, int team_id) {
  EpsSmem s;
  const size_t region = stream_bytes(a.stream_stages);
  const size_t img_bytes = a.table_global ? region * a.teams : a.image_bytes;
  s.img = smem;
  s.stream = smem + region * team_id;
  s.mbar = reinterpret_cast<uint64_t*>(smem + img_bytes);
  EpsCtrl* ctrl = reinterpret_cast<EpsCtrl*>(smem + img_bytes + 16);
  s.sc = ctrl + team_id;
  const int tw16 = (a.track_words + 3) & ~3;
  uint32_t* track_base =
      reinterpret_cast<uint32_t*>(smem + img_bytes + 16 + sizeof(EpsCtrl) * a.teams);
  s.track = track_base + static_cast<size_t>(tw16) * team_id;
  int2* st_base = reinterpret_cast<int2*>(track_base + static_cast<size_t>(tw16) * a.teams);
  s.st = st_base + static_cast<size_t>(team_id) * a.n_slots;
  uint32_t* x_base = reinterpret_cast<uint32_t*>(st_base + static_cast<size_t>(a.teams) * a.n_slots);
  s.X = x_base + static_cast<size_t>(team_id) * a.x_words;
  return s;
}

__device__ __forceinline__ Team eps_team(const EpsArgs& a, int team_id) {
  Team tm;
  tm.tid = threadIdx.x - team_id * a.team_size;
  tm.nthr = a.team_size;
  tm.bar = 1 + team_id;
  tm.lane = threadIdx.x & 31;
  tm.warp = tm.tid >> 5;
  tm.nwarps = a.team_size >> 5;
  return tm;
}

// One breadth-first level: every input path is propagated once; failures
// and solutions are counted; every other node pushes its two children
// (left ub <= m, right lb >= m + 1) to the output level.
template <bool kTrack, bool kLearned, bool kGlobal, bool kStream>
__global__ void __launch_bounds__(1024) k_eps_expand(EpsArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int team_id = threadIdx.x / a.team_size;
  const EpsSmem sm = eps_smem(smem, a, team_id);
  if (!kGlobal) {
    if (threadIdx.x == 0) mbar_init(sm.mbar, 1);
    if (!load_image(sm.img, a.image, a.image_bytes, sm.mbar, 0)) {
      if (threadIdx.x == 0) atomicExch(&a.g->error, 3);
      return;
    }
  }
  if (threadIdx.x == 0 && blockIdx.x == 0 && a.g->t0 == 0)
    atomicCAS(&a.g->t0, 0ull, static_cast<unsigned long long>(eps_now_ns()));
  const Team tm = eps_team(a, team_id);
  const Tab tb = make_tab(kGlobal ? a.image : sm.img, a.levels & (kGlobal ? 2 : 1));
  const Track tk = make_track(sm.track, tb.n_vars, tb.n_lin + tb.n_lin_long);
  const int team_gid = blockIdx.x * a.teams + team_id;
  Streamer stream;
  if (kStream)  // published by the barrier at the top of the work loop
    stream = stream_open(sm.stream, a.stream_stages, tb, a.image, tm, 0u);
  EpsCtrl* sc = sm.sc;
  unsigned long long nodes = 0, published = 0, fails = 0, sols = 0, iters = 0, evals = 0;
  int max_d = 0;
  unsigned par = 0;
  for (;;) {
    if (tm.tid == 0) sc->next = atomicAdd(a.in_counter, 1);
    team_bar(tm.bar, tm.nthr);
    const int p = sc->next;
    if (p >= a.n_in) break;
    const int2* path = a.in_paths + static_cast<size_t>(p) * a.in_len;
    eps_restore<kTrack>(a.root, sm.st, tm, a.n_vars, a.n_slots, tk, path, a.in_len);
    int it = 0;
    unsigned long long key = 0;
    const int r = eps_node<kTrack, kLearned, kGlobal, kStream>(tb, sm.st, tm, sc, tk, false, par, a, it,
                                                                 key, a.in_len, sm.X, &stream);
    par ^= 1u;
    if (r == kNodeStop) break;
    if (tm.tid == 0) {
      eps_count_node(a, nodes, published);
      iters += it;
      evals += sc->fc.evals;
      max_d = max(max_d, a.in_len);
    }
    if (r == kNodeError) {
      if (tm.tid == 0) atomicExch(&a.g->error, 1);
      break;
    }
    if (r == kNodeFailed) {
      if (tm.tid == 0) ++fails;
      continue;
    }
    if (r == kNodeSolution) {
      eps_solution(tb, sm.st, tm, sc, a, team_gid, sols);
      continue;
    }
    // branch: two children appended to the next level
    if (tm.tid == 0) {
      const int o = atomicAdd(a.out_count, 2);
      if (o + 2 > a.out_cap) {
        atomicExch(&a.g->error, 4);
        sc->out = -1;
      } else {
        const int v = tb.branch[static_cast<int>(key & 0xffffffffull)];
        const int2 D = sm.st[v];
        const int m = D.x + (D.y - D.x) / 2;
        const size_t w = static_cast<size_t>(a.in_len) + 1;
        a.out_paths[static_cast<size_t>(o) * w + a.in_len] = make_int2(v, m);
        a.out_paths[static_cast<size_t>(o + 1) * w + a.in_len] =
            make_int2(static_cast<int>(static_cast<uint32_t>(v) | 0x80000000u), m + 1);
        sc->out = o;
      }
    }
    team_bar(tm.bar, tm.nthr);
    const int o = sc->out;
    if (o < 0) break;
    const size_t w = static_cast<size_t>(a.in_len) + 1;
    for (int k = tm.tid; k < a.in_len; k += tm.nthr) {
      const int2 e = path[k];
      a.out_paths[static_cast<size_t>(o) * w + k] = e;
      a.out_paths[static_cast<size_t>(o + 1) * w + k] = e;
    }
  }
  // every exit follows a team barrier after the team's last segment
  if (kStream) stream_close(stream);
  if (tm.tid == 0) {
    atomicAdd(&a.g->nodes, nodes);
    atomicAdd(&a.g->fails, fails);
    atomicAdd(&a.g->solutions, sols);
    atomicAdd(&a.g->iterations, iters);
    atomicAdd(&a.g->evals, evals);
    atomicMax(&a.g->max_depth, max_d);
  }
}

// Persistent teams search the subtrees under the frontier paths depth first.
template <bool kTrack, bool kLearned, bool kGlobal, bool kStream>
__global__ void __launch_bounds__(1024) k_eps_solve(EpsArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int team_id = threadIdx.x / a.team_size;
  const EpsSmem sm = eps_smem(smem, a, team_id);
  if (!kGlobal) {
    if (threadIdx.x == 0) mbar_init(sm.mbar, 1);
    if (!load_image(sm.img, a.image, a.image_bytes, sm.mbar, 0)) {
      if (threadIdx.x == 0) atomicExch(&a.g->error, 3);
      return;
    }
  }
  if (threadIdx.x == 0 && blockIdx.x == 0 && a.g->t0 == 0)
    atomicCAS(&a.g->t0, 0ull, static_cast<unsigned long long>(eps_now_ns()));
  const Team tm = eps_team(a, team_id);
  const Tab tb = make_tab(kGlobal ? a.image : sm.img, a.levels & (kGlobal ? 2 : 1));
  const Track tk = make_track(sm.track, tb.n_vars, tb.n_lin + tb.n_lin_long);
  const int team_gid = blockIdx.x * a.teams + team_id;
  Streamer stream;
  if (kStream)  // published by the barrier at the top of the work loop
    stream = stream_open(sm.stream, a.stream_stages, tb, a.image, tm, 0u);
  EpsCtrl* sc = sm.sc;
  int2* stack = a.stacks + static_cast<size_t>(team_gid) * a.max_depth;
  const int base = a.in_len;
  unsigned long long nodes = 0, published = 0, fails = 0, sols = 0, iters = 0, evals = 0;
  int max_d = 0;
  unsigned par = 0;
  bool done = false;
  while (!done) {
    if (tm.tid == 0) sc->next = atomicAdd(a.in_counter, 1);
    team_bar(tm.bar, tm.nthr);
    const int p = sc->next;
    if (p >= a.n_in) break;
    const int2* path = a.in_paths + static_cast<size_t>(p) * base;
    for (int k = tm.tid; k < base; k += tm.nthr) stack[k] = path[k];
    int depth = base;  // thread 0's copy is authoritative
    eps_restore<kTrack>(a.root, sm.st, tm, a.n_vars, a.n_slots, tk, path, base);
    bool seeded = false;  // team-uniform
    for (;;) {
      int it = 0;
      unsigned long long key = 0;
      const int r = eps_node<kTrack, kLearned, kGlobal, kStream>(tb, sm.st, tm, sc, tk, seeded, par, a,
                                                                   it, key, depth, sm.X, &stream);
      par ^= 1u;
      if (r == kNodeStop) {
        done = true;
        break;
      }
      if (tm.tid == 0) {
        eps_count_node(a, nodes, published);
        iters += it;
        evals += sc->fc.evals;
        max_d = max(max_d, depth);
      }
      if (r == kNodeError) {
        if (tm.tid == 0) atomicExch(&a.g->error, 1);
        done = true;
        break;
      }
      if (r == kNodeBranch) {
        if (tm.tid == 0) {
          int err = 0;
          if (depth >= a.max_depth) {
            err = 1;
            atomicExch(&a.g->error, 2);
          } else {
            const int v = tb.branch[static_cast<int>(key & 0xffffffffull)];
            const int2 D = sm.st[v];
            const int m = D.x + (D.y - D.x) / 2;
            stack[depth] = make_int2(v, m);
            ++depth;
            atom_min_s32(&sm.st[v].y, m);  // m < ub(v): always a change
            if (kTrack) mark_changed(tb, tk, 2, v);
          }
          sc->err = err;
        }
        team_bar(tm.bar, tm.nthr);
        if (sc->err) {
          done = true;
          break;
        }
        seeded = true;
        continue;
      }
      if (r == kNodeFailed) {
        if (tm.tid == 0) ++fails;
      } else {
        eps_solution(tb, sm.st, tm, sc, a, team_gid, sols);
      }
      // backtrack within the subtree: never above the subproblem's path
      if (tm.tid == 0) {
        while (depth > base && (static_cast<uint32_t>(stack[depth - 1].x) & 0x80000000u)) --depth;
        if (depth == base) {
          sc->depth = -1;
        } else {
          const int2 e = stack[depth - 1];
          stack[depth - 1] =
              make_int2(static_cast<int>(static_cast<uint32_t>(e.x) | 0x80000000u), e.y + 1);
          sc->depth = depth;
        }
      }
      team_bar(tm.bar, tm.nthr);
      const int d = sc->depth;
      if (d < 0) break;  // subtree exhausted: next subproblem
      eps_restore<kTrack>(a.root, sm.st, tm, a.n_vars, a.n_slots, tk, stack, d);
      seeded = false;
    }
  }
  // every exit follows a team barrier after the team's last segment
  if (kStream) stream_close(stream);
  if (tm.tid == 0) {
    atomicAdd(&a.g->nodes, nodes);
    atomicAdd(&a.g->fails, fails);
    atomicAdd(&a.g->solutions, sols);
    atomicAdd(&a.g->iterations, iters);
    atomicAdd(&a.g->evals, evals);
    atomicMax(&a.g->max_depth, max_d);
  }
}

}  // namespace pccp
