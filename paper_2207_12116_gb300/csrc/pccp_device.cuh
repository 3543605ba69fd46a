// pccp_device.cuh -- device-side building blocks of the propagation fixed point.
//
// A "team" is a group of whole warps (32..1024 threads) that owns one store of
// intervals in shared memory and evaluates every propagator row of the model
// on it, concurrently and without locks (Sec. 4 load/store semantics; Sec. 5
// fixed-point loop).  Every tell is a lattice join done by an atomic max on a
// lower bound or an atomic min on an upper bound (the join of ZInc / ZDec,
// Sec. 2).  A tell is only issued when the candidate is strictly stronger
// than the value the thread loaded (the "store only if ox > rx" rule of the
// Sec. 4 compilation), and reads of shared bounds are relaxed atomic loads
// (the ATOM requirement of Sec. 4 and the erratum of Sec. 5).  Teams
// synchronise on a named barrier whose OR-reduction both ends an iteration
// and detects the fixed point (the has_changed flags of Sec. 5).
#pragma once

#include <cstdint>

namespace pccp {

enum : int { kFixpoint = 0, kFailed = 1, kError = 2 };

// Header at the start of the packed table image (128 bytes).  The image is
// copied verbatim into shared memory, so every offset is relative to its start
// and 16-byte aligned.
struct TableHeader {
  int32_t n_vars, n_t, n_rf, n_lin, n_terms, n_branch, objective, image_bytes;
  int32_t off_t, off_rf, off_lin, off_terms, off_branch, n_lin_long, off_lin_long, off_terms_long;
  int32_t off_adj_off, off_adj, n_adj, off_bstat, off_rfp, n_rfp;
  int32_t rows_sweep;   // row evaluations in one full sweep (a reified pair counts 2)
  int32_t bytes_sweep;  // their algorithmic bytes
  int32_t off_seg, n_seg;  // stream segments (tables read from global memory)
  // prefixes of the image that a kernel copies into shared memory: core_bytes
  // (header, rows, branch variables, their static features) without change
  // tracking, track_bytes (also the variable -> linear-row adjacency) with it;
  // the stream segment list after them is only read from global memory
  int32_t core_bytes, track_bytes;
  // store layout: variables 0 .. bit0-1 as int2 {lb, ub} slots; variables
  // bit0 .. n_vars-1 (Booleans, when the model keeps them as bits) 32 to a
  // slot {lb bits, ub bits}; n_slots = bit0 + ceil((n_vars - bit0) / 32)
  int32_t bit0, n_slots;
  // temporal rows in topological levels (n_tlev > 0 when the rows x + d <= y
  // form an acyclic graph over the variables): int32 level bounds
  // [n_tlev + 1] at off_tlev, then (16-byte aligned) the rows grouped by the
  // level of x, the length of the longest chain of rows ending at x
  int32_t off_tlev, n_tlev;
};
static_assert(sizeof(TableHeader) == 128, "header must be 128 bytes");

// Streamed tables.  When a table does not fit in shared memory beside a store,
// a sweep brings its rows in as a cyclic sequence of segments of at most
// kStreamChunk bytes, each a byte range of the image holding whole rows of one
// kind, copied by TMA bulk copies into a ring of per-team buffers.
constexpr int kStreamChunk = 32768;
constexpr int kStreamMaxStages = 3;
enum : int32_t {
  kSegPairs = 0,      // reified pairs (uint4)
  kSegSingles = 1,    // single reified rows (uint2)
  kSegTemporal = 2,   // temporal rows (uint2)
  kSegShort = 3,      // whole tiles of short linear rows: their terms
  kSegLong = 4,       // whole long linear rows: their terms
  kSegLongGlobal = 5  // long rows longer than a chunk: terms read from global memory
};
struct StreamSeg {
  int32_t kind, first, count;  // rows first .. first + count - 1 of that kind
  int32_t src_off, bytes;      // byte range of the image (16-byte aligned; bytes may be 0)
  int32_t term_base;           // kSegShort / kSegLong: term index at src_off
  int32_t pad[2];
};
static_assert(sizeof(StreamSeg) == 32, "segment record must be 32 bytes");

// Row encodings (structure of arrays, one array per row kind):
//   temporal  uint2 {x | y << 16, d}              x + d <= y
//   reified   uint2 {x | y << 16, b | d << 16}    b <=> (x <= y && y < x + d), d int16
//   linear    int4  {c, base, len, flags}         sum coef*var <= c; flags: 1 all coef > 0,
//                                                 2 and all vars 0/1 at the root
//   term      uint32 var | coef << 16             coef int16
// Linear rows of at most kShortRow terms are evaluated by one thread each and
// stored in tiles of 32 rows, transposed: term t of the row in lane l of a
// tile sits at base + 32 t, base = tile start + l, so the 32 lanes of a warp
// read 32 consecutive words.  Longer rows are evaluated by a warp each and
// stored row-major (term k at base + k).
constexpr int kShortRow = 64;

struct Tab {
  const uint2* t;
  const uint2* rf;
  const uint4* rfp;         // reified pairs {x | y << 16, b1 | d1 << 16, b2 | d2 << 16, 0}
  const int4* lin;          // short rows
  const uint32_t* terms;    // their tiled terms
  const int4* lin_long;     // long rows
  const uint32_t* terms_long;
  const int32_t* branch;
  const int32_t* adj_off;   // [n_vars + 1]: linear rows holding each variable
  const int32_t* adj;       // row ids: short rows 0.., long rows n_lin..
  const float* bstat;       // [n_branch][8] static features of the branch variables
  int n_vars, n_t, n_rf, n_rfp, n_lin, n_lin_long, n_terms, n_branch, objective;
  int rows_sweep, bytes_sweep;
  const StreamSeg* seg;
  int n_seg;
  int bit0, n_slots;  // store layout (see TableHeader)
  const int32_t* tlev_off;  // temporal rows in levels (see TableHeader); n_tlev 0: none
  const uint2* tlev;
  int n_tlev;
  // short linear rows evaluated by groups of 2^lin_shift lanes (sweeps
  // compiled with kSplit only; 0: a thread per row)
  int lin_shift;
};

__host__ __device__ __forceinline__ int align16_dev(int x) { return (x + 15) & ~15; }

__device__ __forceinline__ Tab make_tab(const uint8_t* img) {
  const TableHeader* h = reinterpret_cast<const TableHeader*>(img);
  Tab tb;
  tb.n_vars = h->n_vars;
  tb.n_t = h->n_t;
  tb.n_rf = h->n_rf;
  tb.n_lin = h->n_lin;
  tb.n_terms = h->n_terms;
  tb.n_branch = h->n_branch;
  tb.objective = h->objective;
  tb.t = reinterpret_cast<const uint2*>(img + h->off_t);
  tb.rf = reinterpret_cast<const uint2*>(img + h->off_rf);
  tb.lin = reinterpret_cast<const int4*>(img + h->off_lin);
  tb.terms = reinterpret_cast<const uint32_t*>(img + h->off_terms);
  tb.n_lin_long = h->n_lin_long;
  tb.lin_shift = 0;
  tb.lin_long = reinterpret_cast<const int4*>(img + h->off_lin_long);
  tb.terms_long = reinterpret_cast<const uint32_t*>(img + h->off_terms_long);
  tb.branch = reinterpret_cast<const int32_t*>(img + h->off_branch);
  tb.adj_off = reinterpret_cast<const int32_t*>(img + h->off_adj_off);
  tb.adj = reinterpret_cast<const int32_t*>(img + h->off_adj);
  tb.bstat = reinterpret_cast<const float*>(img + h->off_bstat);
  tb.n_rfp = h->n_rfp;
  tb.rows_sweep = h->rows_sweep;
  tb.bytes_sweep = h->bytes_sweep;
  tb.seg = reinterpret_cast<const StreamSeg*>(img + h->off_seg);
  tb.n_seg = h->n_seg;
  tb.rfp = reinterpret_cast<const uint4*>(img + h->off_rfp);
  tb.bit0 = h->bit0;
  tb.n_slots = h->n_slots;
  tb.n_tlev = h->n_tlev;
  tb.tlev_off = reinterpret_cast<const int32_t*>(img + h->off_tlev);
  tb.tlev = reinterpret_cast<const uint2*>(img + align16_dev(h->off_tlev + 4 * (h->n_tlev + 1)));
  return tb;
}

// The same with the temporal levels used only when `levels` is non-zero.
__device__ __forceinline__ Tab make_tab(const uint8_t* img, int levels) {
  Tab tb = make_tab(img);
  if (!levels) tb.n_tlev = 0;
  return tb;
}

// Point tb's temporal levels at a copy of their section (at p, 16-byte aligned).
__device__ __forceinline__ void tab_levels_at(Tab& tb, const uint8_t* p) {
  tb.tlev_off = reinterpret_cast<const int32_t*>(p);
  tb.tlev = reinterpret_cast<const uint2*>(p + align16_dev(4 * (tb.n_tlev + 1)));
}

// ------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Relaxed, CTA-scope load of the interval {lb, ub} of variable v.  Each 32-bit
// element is a single-copy-atomic access; lb and ub are independent lattice
// components so they need not be read together.
__device__ __forceinline__ int2 ld_dom(const int2* st, int v) {
  int2 r;
  asm volatile("ld.relaxed.cta.shared::cta.v2.s32 {%0, %1}, [%2];"
               : "=r"(r.x), "=r"(r.y)
               : "r"(smem_u32(st + v)));
  return r;
}

__device__ __forceinline__ int atom_max_s32(int* p, int v) {
  int old;
  asm volatile("atom.relaxed.cta.shared::cta.max.s32 %0, [%1], %2;"
               : "=r"(old)
               : "r"(smem_u32(p)), "r"(v)
               : "memory");
  return old;
}

__device__ __forceinline__ int atom_min_s32(int* p, int v) {
  int old;
  asm volatile("atom.relaxed.cta.shared::cta.min.s32 %0, [%1], %2;"
               : "=r"(old)
               : "r"(smem_u32(p)), "r"(v)
               : "memory");
  return old;
}

// The same joins without the old value (the caller knows from its snapshot
// that the bound moves, unless another thread moved it further meanwhile).
__device__ __forceinline__ void red_max_s32(int* p, int v) {
  asm volatile("red.relaxed.cta.shared::cta.max.s32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v)
               : "memory");
}

__device__ __forceinline__ void red_min_s32(int* p, int v) {
  asm volatile("red.relaxed.cta.shared::cta.min.s32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v)
               : "memory");
}

// Relaxed CTA-scope shared atomic OR / AND returning the old word (the joins
// of a slot of Booleans: OR raises lower bounds, AND lowers upper bounds).
__device__ __forceinline__ uint32_t atom_or_old(int* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.relaxed.cta.shared::cta.or.b32 %0, [%1], %2;"
               : "=r"(old)
               : "r"(smem_u32(p)), "r"(v)
               : "memory");
  return old;
}

__device__ __forceinline__ uint32_t atom_and_old(int* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.relaxed.cta.shared::cta.and.b32 %0, [%1], %2;"
               : "=r"(old)
               : "r"(smem_u32(p)), "r"(v)
               : "memory");
  return old;
}

// Domain of variable v in a store of either layout: an int2 slot below bit0,
// else bit (v - bit0) % 32 of slot bit0 + (v - bit0) / 32, lower bounds in the
// slot's first word and upper bounds in its second (one 8-byte relaxed load
// either way).
// kBits = false (kernels for tables staged in shared memory, whose models
// never keep bits): a plain interval load.
template <bool kBits = true>
__device__ __forceinline__ int2 ld_var(const int2* st, int bit0, int v) {
  if (!kBits || v < bit0) return ld_dom(st, v);
  const int q = v - bit0;
  const int2 W = ld_dom(st, bit0 + (q >> 5));
  return make_int2((W.x >> (q & 31)) & 1, (W.y >> (q & 31)) & 1);
}

// Value of variable v (its lower bound) for witnesses and write-back.
__device__ __forceinline__ int2 var_dom_plain(const int2* st, int bit0, int v) {
  if (v < bit0) return st[v];
  const int q = v - bit0;
  const int2 W = st[bit0 + (q >> 5)];
  return make_int2((W.x >> (q & 31)) & 1, (W.y >> (q & 31)) & 1);
}

// Emptiness of one store slot (an interval, or 32 Booleans).
__device__ __forceinline__ bool slot_empty(int2 D, int slot, int bit0) {
  return slot < bit0 ? D.x > D.y : (static_cast<uint32_t>(D.x) & ~static_cast<uint32_t>(D.y)) != 0u;
}

__device__ __forceinline__ void st_relaxed(int* p, int v) {
  asm volatile("st.relaxed.cta.shared::cta.s32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.cta.shared::cta.s32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}

// Named barrier over `n` threads (a multiple of 32) with an OR-reduction of p.
__device__ __forceinline__ bool team_bar_or(int id, int n, bool p) {
  int r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.s32 pi, %1, 0;\n\t"
      "bar.red.or.pred po, %2, %3, pi;\n\t"
      "selp.s32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"(static_cast<int>(p)), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// Named barrier over `n` threads returning how many of them passed p.
__device__ __forceinline__ int team_bar_popc(int id, int n, bool p) {
  int r;
  asm volatile(
      "{\n\t.reg .pred pi;\n\t"
      "setp.ne.s32 pi, %1, 0;\n\t"
      "bar.red.popc.u32 %0, %2, %3, pi;\n\t}"
      : "=r"(r)
      : "r"(static_cast<int>(p)), "r"(id), "r"(n)
      : "memory");
  return r;
}

__device__ __forceinline__ void team_bar(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// ------------------------------------------------------------ mbarrier / TMA bulk copy

__device__ __forceinline__ void mbar_init(uint64_t* mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
               : "memory");
}

// Plain arrive (count 1) on an mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// Make mbarrier initialisation visible to the async proxy (TMA completions).
__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
}

// 1-D TMA bulk copy global -> shared, completing `bytes` on the mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: true when the phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity, int max_tries) {
  for (int i = 0; i < max_tries; ++i)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

// ------------------------------------------------------------ team context

struct Team {
  int tid;     // thread index in the team
  int nthr;    // team size (multiple of 32)
  int bar;     // named barrier id (1..15)
  int lane;
  int warp;    // warp index in the team
  int nwarps;
};

struct Flags {
  bool ch;  // some tell strengthened the store
  bool fl;  // some tell found an empty interval
  int evals;  // rows evaluated by this thread
  int bytes;  // algorithmic bytes read by this thread (rows, bounds, checks)
};

// Change tracking of one team (shared memory).  Three rotating pairs of
// bitmaps (the past / present / future rotation of the has_changed flags of
// Sec. 5): chg marks variables strengthened during an iteration, dl marks
// the linear rows holding such a variable.  Iteration k writes buffer k%3,
// reads buffer (k+2)%3 (the previous iteration's changes) and clears
// buffer (k+1)%3 for the next iteration.  A row whose variables did not
// change since its last evaluation is stable and is skipped: the fixed point
// is unchanged because every row that could still tell something is run
// again after each change of its inputs (the fair-schedule argument of
// Sec. 3).
struct Track {
  uint32_t* chg;  // [3][W]
  uint32_t* dl;   // [3][WL]
  int W, WL;
};

__host__ __device__ __forceinline__ int track_words(int n_vars, int n_lin_rows) {
  return 3 * ((n_vars + 31) / 32) + 3 * ((n_lin_rows + 31) / 32);
}

__device__ __forceinline__ Track make_track(uint32_t* base, int n_vars, int n_lin_rows) {
  Track t;
  t.W = (n_vars + 31) / 32;
  t.WL = (n_lin_rows + 31) / 32;
  t.chg = base;
  t.dl = base + 3 * t.W;
  return t;
}

__device__ __forceinline__ void atom_or_u32(uint32_t* p, uint32_t v) {
  asm volatile("atom.relaxed.cta.shared::cta.or.b32 _, [%0], %1;" ::"r"(smem_u32(p)), "r"(v)
               : "memory");
}

__device__ __forceinline__ bool test_bit(const uint32_t* bm, int i) {
  return (bm[i >> 5] >> (i & 31)) & 1u;
}

// Record that variable v changed in buffer `cur`: its bit, and the dirty
// bits of the linear rows that hold it.
__device__ __forceinline__ void mark_changed(const Tab& tb, const Track& tk, int cur, int v) {
  atom_or_u32(&tk.chg[cur * tk.W + (v >> 5)], 1u << (v & 31));
  for (int k = tb.adj_off[v]; k < tb.adj_off[v + 1]; ++k) {
    const int r = tb.adj[k];
    atom_or_u32(&tk.dl[cur * tk.WL + (r >> 5)], 1u << (r & 31));
  }
}

// floor(a / b) for b > 0.
__device__ __forceinline__ int floor_div_pos(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

// Join cand into lb(v).  lb_seen/ub_seen are the values this thread loaded;
// bounds only move inward, so cand <= lb_seen means the tell is a no-op and
// cand > ub_seen means the interval is empty whatever happened since.
// Context of one sweep: the table, the store, the change tracking, the
// buffer written this iteration and the one read (the previous iteration's
// changes), and whether every row must run (first iteration of a fresh store).
struct Sweep {
  const Tab& tb;
  int2* st;
  const Track& tk;
  int cur;
  const uint32_t* prev_chg;
  const uint32_t* prev_dl;
  bool full;
  int* grab;  // this sweep's claim counter (tables in global memory)
};

template <bool kTrack>
__device__ __forceinline__ void tell_lb(const Sweep& w, int v, int cand, int lb_seen, int ub_seen,
                                        Flags& f) {
  if (cand <= lb_seen) return;
  if (cand > ub_seen) {
    f.fl = true;
    return;
  }
  int old = atom_max_s32(&w.st[v].x, cand);
  if (old < cand) {
    f.ch = true;
    if (kTrack) mark_changed(w.tb, w.tk, w.cur, v);
  }
}

template <bool kTrack>
__device__ __forceinline__ void tell_ub(const Sweep& w, int v, int cand, int lb_seen, int ub_seen,
                                        Flags& f) {
  if (cand >= ub_seen) return;
  if (cand < lb_seen) {
    f.fl = true;
    return;
  }
  int old = atom_min_s32(&w.st[v].y, cand);
  if (old > cand) {
    f.ch = true;
    if (kTrack) mark_changed(w.tb, w.tk, w.cur, v);
  }
}

// Tells on a variable that may be a Boolean kept as bits (the b of a
// reified row, a term of an all-positive 0/1 linear row): candidates are 0 or
// 1 there, so a tell sets the lower bit (OR) or clears the upper bit (AND);
// below bit0 they are the interval tells.
template <bool kTrack, bool kBits>
__device__ __forceinline__ void tell_lb_v(const Sweep& w, int v, int cand, int lb_seen,
                                          int ub_seen, Flags& f) {
  if (!kBits || v < w.tb.bit0) {
    tell_lb<kTrack>(w, v, cand, lb_seen, ub_seen, f);
    return;
  }
  if (cand <= lb_seen) return;
  if (cand > ub_seen) {
    f.fl = true;
    return;
  }
  const int q = v - w.tb.bit0;
  const uint32_t m = 1u << (q & 31);
  if (!(atom_or_old(&w.st[w.tb.bit0 + (q >> 5)].x, m) & m)) {
    f.ch = true;
    if (kTrack) mark_changed(w.tb, w.tk, w.cur, v);
  }
}

template <bool kTrack, bool kBits>
__device__ __forceinline__ void tell_ub_v(const Sweep& w, int v, int cand, int lb_seen,
                                          int ub_seen, Flags& f) {
  if (!kBits || v < w.tb.bit0) {
    tell_ub<kTrack>(w, v, cand, lb_seen, ub_seen, f);
    return;
  }
  if (cand >= ub_seen) return;
  if (cand < lb_seen) {
    f.fl = true;
    return;
  }
  const int q = v - w.tb.bit0;
  const uint32_t m = 1u << (q & 31);
  if (atom_and_old(&w.st[w.tb.bit0 + (q >> 5)].y, ~m) & m) {
    f.ch = true;
    if (kTrack) mark_changed(w.tb, w.tk, w.cur, v);
  }
}

// Temporal row x + d <= y: ub(x) <= ub(y) - d and lb(y) >= lb(x) + d
// (the [[x + y <= c]] compilation of Sec. 2 with y negated).  The common case
// (nothing to tell) costs one branch.
template <bool kTrack>
__device__ __forceinline__ void eval_temporal(const Sweep& w, uint2 row, Flags& f) {
  const int x = row.x & 0xffff, y = row.x >> 16, d = static_cast<int>(row.y);
  if (kTrack && !w.full && !(test_bit(w.prev_chg, x) | test_bit(w.prev_chg, y))) {
    f.bytes += 16;  // row and two change words
    return;
  }
  f.evals += 1;
  f.bytes += 20;
  const int2 X = ld_dom(w.st, x), Y = ld_dom(w.st, y);
  const int cux = Y.y - d, cly = X.x + d;
  if (cux < X.y || cly > Y.x) {
    tell_ub<kTrack>(w, x, cux, X.x, X.y, f);
    tell_lb<kTrack>(w, y, cly, Y.x, Y.y, f);
  }
}

// The temporal rows level by level, by one warp (tb.n_tlev > 0): kUp, lower
// bounds in increasing levels (lb y >= lb x + d); else upper bounds in
// decreasing levels (ub x <= ub y - d).  A level's rows read only variables
// that earlier levels of the pass have finished, so one pass carries a bound
// along a whole chain of rows, where rows evaluated side by side move it one
// row per sweep.  Only the order of evaluation changes: the fixed point is
// the same (Sec. 3).  The next level's first row is loaded ahead.  A warp
// runs it whole (the shuffles need every lane).
template <bool kTrack, bool kUp>
__device__ __forceinline__ void temporal_levels(const Sweep& w, const Team& tm, Flags& f) {
  const Tab& tb = w.tb;
  const int n = tb.n_tlev;
  // level bounds: up to 31 levels held one per lane and read by shuffles
  const bool in_regs = n < 32;
  const int lane_off = in_regs && tm.lane <= n ? tb.tlev_off[tm.lane] : 0;
  auto bound = [&](int l) {
    return in_regs ? __shfl_sync(0xffffffffu, lane_off, l) : tb.tlev_off[l];
  };
  int L = kUp ? 0 : n - 1;
  int lo = bound(L), hi = bound(L + 1);
  uint2 row = lo + tm.lane < hi ? tb.tlev[lo + tm.lane] : make_uint2(0u, 0u);
  for (int k = 0; k < n; ++k) {
    const int Ln = kUp ? L + 1 : L - 1;
    int nlo = 0, nhi = 0;
    uint2 nrow = make_uint2(0u, 0u);
    if (k + 1 < n) {
      nlo = bound(Ln);
      nhi = bound(Ln + 1);
      if (nlo + tm.lane < nhi) nrow = tb.tlev[nlo + tm.lane];
    }
    for (int r = lo + tm.lane; r < hi; r += 32) {
      if (r != lo + tm.lane) row = tb.tlev[r];
      const int x = row.x & 0xffff, y = row.x >> 16, d = static_cast<int>(row.y);
      const int2 X = ld_dom(w.st, x), Y = ld_dom(w.st, y);
      // tells without a returned value, so the next level waits only for
      // the loads; the change they report may also be another thread's
      // (which moved the same bound in this sweep)
      if (kUp) {
        f.evals += 1;  // a row's two rules count as one evaluation
        f.bytes += 20;
        const int c = X.x + d;
        if (c > Y.x) {
          if (c > Y.y) {
            f.fl = true;
          } else {
            red_max_s32(&w.st[y].x, c);
            f.ch = true;
            if (kTrack) mark_changed(w.tb, w.tk, w.cur, y);
          }
        }
      } else {
        const int c = Y.y - d;
        if (c < X.y) {
          if (c < X.x) {
            f.fl = true;
          } else {
            red_min_s32(&w.st[x].y, c);
            f.ch = true;
            if (kTrack) mark_changed(w.tb, w.tk, w.cur, x);
          }
        }
      }
    }
    __syncwarp();
    L = Ln;
    lo = nlo;
    hi = nhi;
    row = nrow;
  }
}

// Temporal rows of a sweep: in levels by the team's last two warps (one
// warp for both passes in a one-warp team) when the table has levels, else
// a thread per row.  Returns after this thread's share.
template <bool kTrack>
__device__ __forceinline__ void sweep_temporal(const Sweep& w, const Team& tm, Flags& f) {
  const Tab& tb = w.tb;
  if (tb.n_tlev > 0) {
    if (tm.warp == tm.nwarps - 1) temporal_levels<kTrack, true>(w, tm, f);
    if (tm.warp == (tm.nwarps > 1 ? tm.nwarps - 2 : 0)) temporal_levels<kTrack, false>(w, tm, f);
  } else {
    for (int r = tm.tid; r < tb.n_t; r += tm.nthr) eval_temporal<kTrack>(w, tb.t[r], f);
  }
}

// One reified row b <=> (A and B), A: x <= y, B: y <= x + d - 1, on a
// snapshot X, Y, B: the four asks of [[phi <=> psi]] (Sec. 2) joined into the
// candidate bounds (nlx .. nub start as the snapshot or earlier candidates).
__device__ __forceinline__ void reified_rule(int2 X, int2 Y, int2 B, int d, int& nlx, int& nux,
                                             int& nly, int& nuy, int& nlb, int& nub) {
  const bool entA = X.y <= Y.x;           // ub x <= lb y
  const bool entB = Y.y <= X.x + d - 1;   // ub y <= lb x + d - 1
  const bool entNA = X.x >= Y.y + 1;      // lb x >= ub y + 1
  const bool entNB = Y.x >= X.y + d;      // lb y >= ub x + d
  if (B.x >= 1) {                         // b entailed: tell A and B
    nux = min(nux, Y.y);
    nly = max(nly, X.x);
    nuy = min(nuy, X.y + d - 1);
    nlx = max(nlx, Y.x - d + 1);
  }
  if (B.y <= 0 && entA) {                 // not b, A holds: tell not B (x + d <= y)
    nly = max(nly, X.x + d);
    nux = min(nux, Y.y - d);
  }
  if (B.y <= 0 && entB) {                 // not b, B holds: tell not A (y + 1 <= x)
    nlx = max(nlx, Y.x + 1);
    nuy = min(nuy, X.y - 1);
  }
  if (entA && entB) nlb = max(nlb, 1);    // A and B entailed: b
  if (entNA || entNB) nub = min(nub, 0);  // not (A and B) entailed: not b
}

// True when a reified rule b <=> (x <= y and y <= x + d - 1) can tell
// nothing on a snapshot with non-empty intervals, given g1 = lb y - ub x and
// g2 = lb x - ub y: b unfixed with neither the conjunction (g1 >= 0,
// g2 >= 1 - d) nor its negation (g2 >= 1 or g1 >= d) entailed; or b = 1 with
// the conjunction entailed; or b = 0 with the negation entailed (every tell
// of the rule is then already implied by the bounds).  Anything else,
// including an empty b, goes through the full rule.
__device__ __forceinline__ bool rule_quiet(int2 B, int g1, int g2, int d) {
  const bool t = g1 >= 0 && g2 >= 1 - d;
  const bool n = g2 >= 1 || g1 >= d;
  return (B.x == 0 && B.y == 1) ? !(t || n) : (B.x == B.y && (B.x == 1 ? t : n));
}

// Reified row, evaluated on one snapshot; the tells (rare once the store
// settles) sit behind one branch.  kQuiet: rows that cannot tell anything
// (rule_quiet) leave before the rule; that pays where loads are slow (tables
// read from global memory) and costs where issue is the limit (tables in
// shared memory), so the kernels for global tables use it.  kBits: the
// model may keep b as a bit (global tables only; else a plain interval load).
template <bool kTrack, bool kQuiet, bool kBits = kQuiet>
__device__ __forceinline__ void eval_reified(const Sweep& w, uint2 row, Flags& f) {
  const int x = row.x & 0xffff, y = row.x >> 16;
  const int b = row.y & 0xffff, d = static_cast<int>(row.y) >> 16;
  if (kTrack && !w.full &&
      !(test_bit(w.prev_chg, x) | test_bit(w.prev_chg, y) | test_bit(w.prev_chg, b))) {
    f.bytes += 20;  // row and three change words
    return;
  }
  f.evals += 1;
  f.bytes += 40;
  const int2 X = ld_dom(w.st, x), Y = ld_dom(w.st, y), B = ld_var<kBits>(w.st, w.tb.bit0, b);
  if (kQuiet && X.x <= X.y && Y.x <= Y.y && rule_quiet(B, Y.x - X.y, X.x - Y.y, d)) return;
  int nlx = X.x, nux = X.y, nly = Y.x, nuy = Y.y, nlb = B.x, nub = B.y;
  reified_rule(X, Y, B, d, nlx, nux, nly, nuy, nlb, nub);
  if (nlx > X.x || nux < X.y || nly > Y.x || nuy < Y.y || nlb > B.x || nub < B.y) {
    tell_lb<kTrack>(w, x, nlx, X.x, X.y, f);
    tell_ub<kTrack>(w, x, nux, X.x, X.y, f);
    tell_lb<kTrack>(w, y, nly, Y.x, Y.y, f);
    tell_ub<kTrack>(w, y, nuy, Y.x, Y.y, f);
    tell_lb_v<kTrack, kBits>(w, b, nlb, B.x, B.y, f);
    tell_ub_v<kTrack, kBits>(w, b, nub, B.x, B.y, f);
  }
}

// Two reified rows over the same pair of variables with the roles swapped,
// b1 <=> (x <= y and y < x + d1) and b2 <=> (y <= x and x < y + d2) (the
// overlap Booleans b_{i,j} and b_{j,i} of the scheduling model): both rules on
// one snapshot, so x and y are loaded once for two rows.
template <bool kTrack, bool kQuiet, bool kBits = kQuiet>
__device__ __forceinline__ void eval_reified_pair(const Sweep& w, uint4 row, Flags& f) {
  const int x = row.x & 0xffff, y = row.x >> 16;
  const int b1 = row.y & 0xffff, d1 = static_cast<int>(row.y) >> 16;
  const int b2 = row.z & 0xffff, d2 = static_cast<int>(row.z) >> 16;
  if (kTrack && !w.full &&
      !(test_bit(w.prev_chg, x) | test_bit(w.prev_chg, y) | test_bit(w.prev_chg, b1) |
        test_bit(w.prev_chg, b2))) {
    f.bytes += 32;  // row and four change words
    return;
  }
  f.evals += 2;
  f.bytes += 80;
  const int2 X = ld_dom(w.st, x), Y = ld_dom(w.st, y);
  const int2 B1 = ld_var<kBits>(w.st, w.tb.bit0, b1), B2 = ld_var<kBits>(w.st, w.tb.bit0, b2);
  if (kQuiet) {  // neither rule can tell anything (rule 2 swaps x and y)
    const int g1 = Y.x - X.y, g2 = X.x - Y.y;
    if (X.x <= X.y && Y.x <= Y.y && rule_quiet(B1, g1, g2, d1) && rule_quiet(B2, g2, g1, d2))
      return;
  }
  int nlx = X.x, nux = X.y, nly = Y.x, nuy = Y.y;
  int nlb1 = B1.x, nub1 = B1.y, nlb2 = B2.x, nub2 = B2.y;
  reified_rule(X, Y, B1, d1, nlx, nux, nly, nuy, nlb1, nub1);
  reified_rule(Y, X, B2, d2, nly, nuy, nlx, nux, nlb2, nub2);
  if (nlx > X.x || nux < X.y || nly > Y.x || nuy < Y.y || nlb1 > B1.x || nub1 < B1.y ||
      nlb2 > B2.x || nub2 < B2.y) {
    tell_lb<kTrack>(w, x, nlx, X.x, X.y, f);
    tell_ub<kTrack>(w, x, nux, X.x, X.y, f);
    tell_lb<kTrack>(w, y, nly, Y.x, Y.y, f);
    tell_ub<kTrack>(w, y, nuy, Y.x, Y.y, f);
    tell_lb_v<kTrack, kBits>(w, b1, nlb1, B1.x, B1.y, f);
    tell_ub_v<kTrack, kBits>(w, b1, nub1, B1.x, B1.y, f);
    tell_lb_v<kTrack, kBits>(w, b2, nlb2, B2.x, B2.y, f);
    tell_ub_v<kTrack, kBits>(w, b2, nub2, B2.x, B2.y, f);
  }
}

// Long linear row sum a_k x_k <= c, one warp per row, lanes over terms.  S is the
// minimum of the whole sum over the box; term k may be bounded by
// slack_k = c - (S - min_k).  If S + (largest span of one term) <= c no term
// can move, so the second pass is skipped.  Terms of the first 32 stay in
// registers; longer rows reload theirs (a fresher bound only weakens the
// tell, which stays sound, and the last iteration sees a stable store).
template <bool kTrack>
__device__ __forceinline__ bool skip_linear_long(const Sweep& w, int r, int lane, Flags& f) {
  if (kTrack && !w.full && !test_bit(w.prev_dl, w.tb.n_lin + r)) {
    if (lane == 0) f.bytes += 4;
    return true;
  }
  return false;
}

// Long row r with header h; its term k at tp[k] (shared or global memory).
template <bool kTrack, bool kBits>
__device__ __forceinline__ void eval_linear_warp_at(const Sweep& w, int4 h,
                                                    const uint32_t* __restrict__ tp, int lane,
                                                    Flags& f) {
  int2* st = w.st;
  if (lane == 0) {
    f.evals += 1;
    f.bytes += 12 + 12 * h.z;
  }
  const int c = h.x, len = h.z;
  int S = 0, span = 0;
  int v0 = 0, a0 = 0;
  int2 D0 = make_int2(0, 0);
  const bool pos = h.w & 1;  // every coefficient positive: no sign selects
  for (int k = lane; k < len; k += 32) {
    const uint32_t t = tp[k];
    const int v = t & 0xffff, a = static_cast<int>(t) >> 16;
    const int2 D = ld_var<kBits>(st, w.tb.bit0, v);
    const int mt = (pos || a > 0) ? a * D.x : a * D.y;
    const int sp = (pos || a > 0) ? a * (D.y - D.x) : a * (D.x - D.y);
    S += mt;
    span = max(span, sp);
    if (k < 32) {
      v0 = v;
      a0 = a;
      D0 = D;
    }
  }
  S = __reduce_add_sync(0xffffffffu, S);
  span = __reduce_max_sync(0xffffffffu, span);
  if (S > c) {  // even the smallest sum exceeds c
    f.fl = true;
    return;
  }
  if (S + span <= c) return;
  if (h.w & 2) {  // 0/1 variables: as in eval_linear_thread_at
    const int slack0 = c - S;
    for (int k = lane; k < len; k += 32) {
      int v;
      int2 D;
      if (k < 32) {
        if (a0 <= slack0) continue;
        v = v0;
        D = D0;
      } else {
        const uint32_t t = tp[k];
        if ((static_cast<int>(t) >> 16) <= slack0) continue;
        v = t & 0xffff;
        D = ld_var<kBits>(st, w.tb.bit0, v);
      }
      if (D.x == 0 && D.y == 1) tell_ub_v<kTrack, kBits>(w, v, 0, D.x, D.y, f);
    }
    return;
  }
  for (int k = lane; k < len; k += 32) {
    int v, a;
    int2 D;
    if (k < 32) {
      v = v0;
      a = a0;
      D = D0;
    } else {
      const uint32_t t = tp[k];
      v = t & 0xffff;
      a = static_cast<int>(t) >> 16;
      D = ld_var<kBits>(st, w.tb.bit0, v);
    }
    const int mt = a > 0 ? a * D.x : a * D.y;
    const int slack = c - (S - mt);
    if (a > 0) {
      if (a * D.y > slack) tell_ub<kTrack>(w, v, floor_div_pos(slack, a), D.x, D.y, f);
    } else {
      // a x <= slack with a < 0: x >= ceil(slack / a) = -floor(slack / -a)
      if (a * D.x > slack) tell_lb<kTrack>(w, v, -floor_div_pos(slack, -a), D.x, D.y, f);
    }
  }
}

// Short linear row sum a_k x_k <= c evaluated by one thread: the same two
// passes as eval_linear_warp with the sum kept in a register (no warp
// reduction and no idle lanes on rows shorter than a warp).
template <bool kTrack>
__device__ __forceinline__ bool skip_linear_short(const Sweep& w, int r, Flags& f) {
  if (kTrack && !w.full && !test_bit(w.prev_dl, r)) {
    f.bytes += 4;
    return true;
  }
  return false;
}

// Short row with header h; its term k at tp[32 k] (shared or global memory).
template <bool kTrack, bool kBits>
__device__ __forceinline__ void eval_linear_thread_at(const Sweep& w, int4 h,
                                                      const uint32_t* __restrict__ tp, Flags& f) {
  int2* st = w.st;
  const int c = h.x, len = h.z;
  f.evals += 1;
  f.bytes += 12 + 12 * len;
  int S = 0, span = 0;
  if (h.w & 1) {  // every coefficient positive: no sign selects
#pragma unroll 4
    for (int k = 0; k < len; ++k) {
      const uint32_t t = tp[32 * k];
      const int a = static_cast<int>(t) >> 16;
      const int2 D = ld_var<kBits>(st, w.tb.bit0, t & 0xffff);
      S += a * D.x;
      span = max(span, a * (D.y - D.x));
    }
  } else {
#pragma unroll 4
    for (int k = 0; k < len; ++k) {
      const uint32_t t = tp[32 * k];
      const int v = t & 0xffff, a = static_cast<int>(t) >> 16;
      const int2 D = ld_var<kBits>(st, w.tb.bit0, v);
      S += a > 0 ? a * D.x : a * D.y;
      span = max(span, a > 0 ? a * (D.y - D.x) : a * (D.x - D.y));
    }
  }
  if (S > c) {
    f.fl = true;
    return;
  }
  if (S + span <= c) return;
  if (h.w & 2) {
    // positive coefficients over 0/1 variables: with slack0 = c - S, term k
    // moves iff a * (ub - lb) > slack0, i.e. iff it is [0, 1] and a > slack0,
    // and then to floor(slack0 / a) = 0.  The coefficient test comes first,
    // so terms that cannot move skip their interval load.
    const int slack0 = c - S;
    for (int k = 0; k < len; ++k) {
      const uint32_t t = tp[32 * k];
      if ((static_cast<int>(t) >> 16) <= slack0) continue;
      const int v = t & 0xffff;
      const int2 D = ld_var<kBits>(st, w.tb.bit0, v);
      if (D.x == 0 && D.y == 1) tell_ub_v<kTrack, kBits>(w, v, 0, D.x, D.y, f);
    }
    return;
  }
  for (int k = 0; k < len; ++k) {
    const uint32_t t = tp[32 * k];
    const int v = t & 0xffff, a = static_cast<int>(t) >> 16;
    const int2 D = ld_var<kBits>(st, w.tb.bit0, v);
    const int mt = a > 0 ? a * D.x : a * D.y;
    const int slack = c - (S - mt);
    if (a > 0) {
      if (a * D.y > slack) tell_ub<kTrack>(w, v, floor_div_pos(slack, a), D.x, D.y, f);
    } else {
      if (a * D.x > slack) tell_lb<kTrack>(w, v, -floor_div_pos(slack, -a), D.x, D.y, f);
    }
  }
}

// Short row with header h evaluated by a group of G = 2^gs consecutive lanes
// (lane j of the group takes terms j, j + G, ...): the sums of eval_linear_
// thread_at reduced over the group by shuffles, then each lane tells its own
// terms.  A row's chain of dependent loads shrinks G-fold, which pays where
// one team's sweep waits on its longest row (a depth-first search alone on an
// SM); every lane of a group computes the same S, so the tells are those of
// the one-thread evaluation.  The group's terms share the row's bank of the
// transposed tile (G-way bank conflicts on the term loads).
template <bool kTrack>
__device__ __forceinline__ void eval_linear_group_at(const Sweep& w, int4 h,
                                                     const uint32_t* __restrict__ tp, int j,
                                                     int gs, Flags& f) {
  int2* st = w.st;
  const int c = h.x, len = h.z, G = 1 << gs;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned gmask = ((1u << G) - 1u) << (lane & ~static_cast<unsigned>(G - 1));
  if (j == 0) {
    f.evals += 1;
    f.bytes += 12 + 12 * len;
  }
  const bool pos = h.w & 1;
  int S = 0, span = 0;
#pragma unroll 4
  for (int k = j; k < len; k += G) {
    const uint32_t t = tp[32 * k];
    const int v = t & 0xffff, a = static_cast<int>(t) >> 16;
    const int2 D = ld_var<false>(st, 0, v);
    S += (pos || a > 0) ? a * D.x : a * D.y;
    span = max(span, (pos || a > 0) ? a * (D.y - D.x) : a * (D.x - D.y));
  }
  for (int o = 1; o < G; o <<= 1) {
    S += __shfl_xor_sync(gmask, S, o);
    span = max(span, __shfl_xor_sync(gmask, span, o));
  }
  if (S > c) {
    f.fl = true;
    return;
  }
  if (S + span <= c) return;
  if (h.w & 2) {  // 0/1 variables: as in eval_linear_thread_at
    const int slack0 = c - S;
    for (int k = j; k < len; k += G) {
      const uint32_t t = tp[32 * k];
      if ((static_cast<int>(t) >> 16) <= slack0) continue;
      const int v = t & 0xffff;
      const int2 D = ld_var<false>(st, 0, v);
      if (D.x == 0 && D.y == 1) tell_ub_v<kTrack, false>(w, v, 0, D.x, D.y, f);
    }
    return;
  }
  for (int k = j; k < len; k += G) {
    const uint32_t t = tp[32 * k];
    const int v = t & 0xffff, a = static_cast<int>(t) >> 16;
    const int2 D = ld_var<false>(st, 0, v);
    const int mt = a > 0 ? a * D.x : a * D.y;
    const int slack = c - (S - mt);
    if (a > 0) {
      if (a * D.y > slack) tell_ub<kTrack>(w, v, floor_div_pos(slack, a), D.x, D.y, f);
    } else {
      if (a * D.x > slack) tell_lb<kTrack>(w, v, -floor_div_pos(slack, -a), D.x, D.y, f);
    }
  }
}

// The lane-group shift for short linear rows of a team of nthr threads: the
// largest G = 2^s <= 8 with G lanes for every row and at least 6 terms per
// lane on the longest row (rows are stored longest first).
__device__ __forceinline__ int lin_split_shift(const Tab& tb, int nthr) {
  if (tb.n_lin <= 0) return 0;
  const int len0 = tb.lin[0].z;
  int s = 0;
  while (s < 3 && (tb.n_lin << (s + 1)) <= nthr && (len0 >> (s + 1)) >= 6) ++s;
  return s;
}

// One full evaluation of every row of the table (one iteration of the
// eventless loop).  Rows of one kind run back to back so warps stay uniform:
// a thread per reified, temporal and short linear row, a warp per long
// linear row; dealt statically, except that with the table in global memory
// warps claim the long rows and the reified pairs (w.grab).  Kind order (it never changes the fixed point, Sec. 3): with
// the table in shared memory reified, temporal, linear; in global memory
// linear, reified, temporal -- each the faster of the six orders measured
// there (the second saves iterations on 120-task models, the first is
// faster for the depth-first searches of 30-task models).  kBits: the model
// keeps Booleans as bits (global tables only).
template <bool kTrack, bool kQuiet, bool kBits, bool kSplit = false>
__device__ __forceinline__ void sweep_rows(const Sweep& w, const Team& tm, Flags& f) {
  const Tab& tb = w.tb;
  // the warps that walk the temporal levels then take their share of the
  // other rows too (leaving those to the other warps measured slower)
  const bool lev = tb.n_tlev > 0;
  const Team& dt = tm;
  if (kQuiet) {  // tables in global memory: linear, reified, temporal
    if (lev) sweep_temporal<kTrack>(w, tm, f);  // levels first
    for (int r = dt.tid; r < tb.n_lin; r += dt.nthr) {
      if (skip_linear_short<kTrack>(w, r, f)) continue;
      const int4 h = tb.lin[r];
      eval_linear_thread_at<kTrack, kBits>(w, h, tb.terms + h.y, f);
    }
    // long rows, then blocks of 32 reified pairs, claimed by whole warps from
    // the sweep's counter: rows of uneven cost (lengths, skipped rows, L2
    // latency) leave no warp waiting at the barrier while others still work
    const int n_blocks = (tb.n_rfp + 31) >> 5;
    for (;;) {
      int q = 0;
      if (tm.lane == 0) q = atomicAdd(w.grab, 1);
      q = __shfl_sync(0xffffffffu, q, 0);
      if (q < tb.n_lin_long) {
        if (skip_linear_long<kTrack>(w, q, tm.lane, f)) continue;
        const int4 h = tb.lin_long[q];
        eval_linear_warp_at<kTrack, kBits>(w, h, tb.terms_long + h.y, tm.lane, f);
      } else if (q < tb.n_lin_long + n_blocks) {
        const int r = ((q - tb.n_lin_long) << 5) + tm.lane;
        if (r < tb.n_rfp) eval_reified_pair<kTrack, kQuiet, kBits>(w, tb.rfp[r], f);
      } else {
        break;
      }
    }
    for (int r = dt.tid; r < tb.n_rf; r += dt.nthr)
      eval_reified<kTrack, kQuiet, kBits>(w, tb.rf[r], f);
    if (!lev) sweep_temporal<kTrack>(w, tm, f);
  } else if (kSplit && !kBits) {
    // tables in shared memory, depth-first searches: the same order, with
    // the table's fields read once into registers (the searches get the
    // table by reference, and the loops' atomics through generic pointers
    // would otherwise make every iteration reload them), and short linear
    // rows by groups of 2^gs consecutive lanes (u = tid + k nthr: a group's
    // lanes share r, so they loop and skip together)
    const uint4* rfp = tb.rfp;
    const uint2* rf = tb.rf;
    const uint2* trow = tb.t;
    const int4* lin = tb.lin;
    const uint32_t* terms = tb.terms;
    const int n_rfp = tb.n_rfp, n_rf = tb.n_rf, n_t = tb.n_t, n_lin = tb.n_lin;
    const int n_lin_long = tb.n_lin_long, gs = tb.lin_shift;
    if (lev) sweep_temporal<kTrack>(w, tm, f);  // levels first
    for (int r = dt.tid; r < n_rfp; r += dt.nthr)
      eval_reified_pair<kTrack, kQuiet, false>(w, rfp[r], f);
    for (int r = dt.tid; r < n_rf; r += dt.nthr) eval_reified<kTrack, kQuiet, false>(w, rf[r], f);
    if (!lev)
      for (int r = dt.tid; r < n_t; r += dt.nthr) eval_temporal<kTrack>(w, trow[r], f);
    if (gs > 0) {
      for (int u = dt.tid; u < (n_lin << gs); u += dt.nthr) {
        const int r = u >> gs;
        if (skip_linear_short<kTrack>(w, r, f)) continue;
        const int4 h = lin[r];
        eval_linear_group_at<kTrack>(w, h, terms + h.y, u & ((1 << gs) - 1), gs, f);
      }
    } else {
      for (int r = dt.tid; r < n_lin; r += dt.nthr) {
        if (skip_linear_short<kTrack>(w, r, f)) continue;
        const int4 h = lin[r];
        eval_linear_thread_at<kTrack, false>(w, h, terms + h.y, f);
      }
    }
    if (n_lin_long > 0) {
      const int4* lin_long = tb.lin_long;
      const uint32_t* terms_long = tb.terms_long;
      for (int r = dt.warp; r < n_lin_long; r += dt.nwarps) {
        if (skip_linear_long<kTrack>(w, r, tm.lane, f)) continue;
        const int4 h = lin_long[r];
        eval_linear_warp_at<kTrack, false>(w, h, terms_long + h.y, tm.lane, f);
      }
    }
  } else {  // tables in shared memory: reified, temporal, linear
    if (lev) sweep_temporal<kTrack>(w, tm, f);  // levels first
    for (int r = dt.tid; r < tb.n_rfp; r += dt.nthr)
      eval_reified_pair<kTrack, kQuiet, kBits>(w, tb.rfp[r], f);
    for (int r = dt.tid; r < tb.n_rf; r += dt.nthr)
      eval_reified<kTrack, kQuiet, kBits>(w, tb.rf[r], f);
    if (!lev) sweep_temporal<kTrack>(w, tm, f);
    for (int r = dt.tid; r < tb.n_lin; r += dt.nthr) {
      if (skip_linear_short<kTrack>(w, r, f)) continue;
      const int4 h = tb.lin[r];
      eval_linear_thread_at<kTrack, kBits>(w, h, tb.terms + h.y, f);
    }
    for (int r = dt.warp; r < tb.n_lin_long; r += dt.nwarps) {
      if (skip_linear_long<kTrack>(w, r, tm.lane, f)) continue;
      const int4 h = tb.lin_long[r];
      eval_linear_warp_at<kTrack, kBits>(w, h, tb.terms_long + h.y, tm.lane, f);
    }
  }
}

// ------------------------------------------------------------ streamed sweep

// Per-team control words of a stream (shared memory, 64 bytes), followed by
// the team's ring of `stages` buffers of kStreamChunk bytes.
struct StreamCtl {
  uint64_t full[kStreamMaxStages];  // phase k of full[b]: the k-th copy into buffer b landed
  uint32_t done[kStreamMaxStages];  // warps finished with the segment in buffer b
  int32_t err;                      // a wait gave up (set by any thread)
  int32_t pad;
};
static_assert(sizeof(StreamCtl) <= 128, "stream control words");
constexpr int kStreamCtlBytes = 128;  // keeps the buffers 128-byte aligned

__host__ __device__ __forceinline__ size_t stream_bytes(int stages) {
  return stages > 0 ? kStreamCtlBytes + static_cast<size_t>(stages) * kStreamChunk : 0;
}

// A team's view of its stream.  g numbers the segments consumed by the team
// since the kernel started (team-uniform: every thread steps it identically);
// segment q is seg[(q - q0) % n_seg] of the image opened at q0, it lands in
// buffer q % stages, and its copy is phase q / stages of that buffer's
// mbarrier.  A sweep consumes exactly n_seg segments, so it starts at
// segment 0.  Invariant between segments: the copies of the next `stages`
// segments have been issued, or will be by the last warp to finish the
// segment before them.
struct Streamer {
  StreamCtl* ctl;
  uint8_t* buf;
  const uint8_t* image;  // device image (global memory)
  const StreamSeg* seg;  // its segment list (global memory)
  int n_seg;
  int stages;
  uint32_t g;
  uint32_t q0;
};

// Wait limit of a stream copy: far above any copy's latency.
constexpr unsigned long long kStreamWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for an mbarrier phase, giving up after kStreamWaitNs of wall time.
__device__ __forceinline__ bool mbar_wait_timed(uint64_t* mbar, uint32_t parity) {
  if (mbar_try_wait(mbar, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(mbar, parity)) return true;
    if (now_ns() - t0 > kStreamWaitNs) return false;
  }
}

// Issue the copy of sequence number q (one thread).
__device__ __forceinline__ void stream_issue(const Streamer& sm, uint32_t q) {
  const StreamSeg s = sm.seg[(q - sm.q0) % static_cast<uint32_t>(sm.n_seg)];
  const int b = static_cast<int>(q % static_cast<uint32_t>(sm.stages));
  uint64_t* mb = &sm.ctl->full[b];
  if (s.bytes > 0) {
    fence_proxy_async_smem();  // earlier generic reads of the buffer come first
    mbar_arrive_expect_tx(mb, static_cast<uint32_t>(s.bytes));
    bulk_copy_g2s(sm.buf + static_cast<size_t>(b) * kStreamChunk, sm.image + s.src_off,
                  static_cast<uint32_t>(s.bytes), mb);
  } else {
    mbar_arrive(mb);  // nothing to copy: complete the phase
  }
}

// Open a stream on an image: thread 0 of the team initialises the control
// words and issues the first `stages` copies.  The caller passes a team
// barrier before any thread consumes a segment.  A stream is closed with
// stream_close before it is reopened or the CTA exits.
__device__ __forceinline__ Streamer stream_open(uint8_t* region, int stages, const Tab& tb,
                                                const uint8_t* image, const Team& tm,
                                                uint32_t g0) {
  Streamer sm;
  sm.ctl = reinterpret_cast<StreamCtl*>(region);
  sm.buf = region + kStreamCtlBytes;
  sm.image = image;
  sm.seg = tb.seg;
  sm.n_seg = tb.n_seg;
  sm.stages = tb.n_seg > 0 ? stages : 0;
  sm.g = g0;
  sm.q0 = g0;
  if (tm.tid == 0 && sm.stages > 0) {
    if (g0 == 0) {
      for (int b = 0; b < kStreamMaxStages; ++b) {
        mbar_init(&sm.ctl->full[b], 1);
        sm.ctl->done[b] = 0u;
      }
      sm.ctl->err = 0;
      fence_mbarrier_init();
    }
    for (int i = 0; i < sm.stages; ++i) stream_issue(sm, sm.g + static_cast<uint32_t>(i));
  }
  return sm;
}

// Wait for the copies still in flight (the next `stages` segments).  Called
// by every thread of the team after a team barrier that follows the last
// segment consumed.  Returns the sequence number to reopen from.
__device__ __forceinline__ uint32_t stream_close(const Streamer& sm) {
  for (int i = 0; i < sm.stages; ++i) {
    const uint32_t q = sm.g + static_cast<uint32_t>(i);
    const int b = static_cast<int>(q % static_cast<uint32_t>(sm.stages));
    if (!mbar_wait_timed(&sm.ctl->full[b], (q / static_cast<uint32_t>(sm.stages)) & 1u))
      sm.ctl->err = 1;
  }
  // the copies of g .. g + stages - 1 were the last phases of the buffers;
  // the next open numbers its segments from there
  return sm.g + static_cast<uint32_t>(sm.stages);
}

// One sweep over a streamed table: the segments in order, each waited for,
// evaluated from its buffer, and released by the last warp to finish it,
// which issues the copy `stages` segments ahead into the freed buffer.
template <bool kTrack>
__device__ __forceinline__ void sweep_rows_streamed(const Sweep& w, const Team& tm, Flags& f,
                                                    Streamer& sm) {
  const Tab& tb = w.tb;
  for (int j = 0; j < sm.n_seg; ++j, ++sm.g) {
    const uint32_t q = sm.g;
    const int b = static_cast<int>(q % static_cast<uint32_t>(sm.stages));
    const StreamSeg s = sm.seg[j];
    const bool ready =
        mbar_wait_timed(&sm.ctl->full[b], (q / static_cast<uint32_t>(sm.stages)) & 1u);
    if (!ready) {
      sm.ctl->err = 1;
    } else {
      const uint8_t* B = sm.buf + static_cast<size_t>(b) * kStreamChunk;
      switch (s.kind) {
        case kSegPairs: {
          const uint4* R = reinterpret_cast<const uint4*>(B);
          for (int i = tm.tid; i < s.count; i += tm.nthr)
            eval_reified_pair<kTrack, true>(w, R[i], f);
          break;
        }
        case kSegSingles: {
          const uint2* R = reinterpret_cast<const uint2*>(B);
          for (int i = tm.tid; i < s.count; i += tm.nthr) eval_reified<kTrack, true>(w, R[i], f);
          break;
        }
        case kSegTemporal: {
          const uint2* R = reinterpret_cast<const uint2*>(B);
          for (int i = tm.tid; i < s.count; i += tm.nthr) eval_temporal<kTrack>(w, R[i], f);
          break;
        }
        case kSegShort: {
          const uint32_t* T = reinterpret_cast<const uint32_t*>(B);
          for (int i = tm.tid; i < s.count; i += tm.nthr) {
            const int r = s.first + i;
            if (skip_linear_short<kTrack>(w, r, f)) continue;
            const int4 h = tb.lin[r];
            eval_linear_thread_at<kTrack, true>(w, h, T + (h.y - s.term_base), f);
          }
          break;
        }
        default: {  // long rows: terms in the buffer, or in global memory
          const bool here = s.kind == kSegLong;
          const uint32_t* T = here ? reinterpret_cast<const uint32_t*>(B) : tb.terms_long;
          const int base = here ? s.term_base : 0;
          for (int i = tm.warp; i < s.count; i += tm.nwarps) {
            const int r = s.first + i;
            if (skip_linear_long<kTrack>(w, r, tm.lane, f)) continue;
            const int4 h = tb.lin_long[r];
            eval_linear_warp_at<kTrack, true>(w, h, T + (h.y - base), tm.lane, f);
          }
          break;
        }
      }
    }
    __syncwarp();
    if (tm.lane == 0) {
      __threadfence_block();  // the warp's reads of the buffer come before its release
      const uint32_t old = atomicAdd(&sm.ctl->done[b], 1u);
      if (old + 1u == static_cast<uint32_t>(tm.nwarps)) {  // last warp: recycle the buffer
        atomicExch(&sm.ctl->done[b], 0u);
        stream_issue(sm, q + static_cast<uint32_t>(sm.stages));
      }
    }
  }
}

// Per-team scalars of the fixed point (shared memory): failure flag and the
// work counters of the current store.
struct FixCtrl {
  int fail;
  int evals;
  int bytes;
  int pad;
  int grab[2];  // claim counters of the sweeps over a table in global memory
  int pad2[2];
};

// Work of `it` full sweeps (every row runs in each, so the count is exact);
// written by the team's thread 0, the only reader of the counters.
template <bool kTrack>
__device__ __forceinline__ void count_sweeps(const Tab& tb, const Team& tm, FixCtrl* fc, int it) {
  if (!kTrack && tm.tid == 0) {
    const long long ev = static_cast<long long>(it) * tb.rows_sweep;
    const long long by = static_cast<long long>(it) * tb.bytes_sweep;
    fc->evals = ev > 0x7fffffffll ? 0x7fffffff : static_cast<int>(ev);
    fc->bytes = by > 0x7fffffffll ? 0x7fffffff : static_cast<int>(by);
  }
}

// Fixed-point loop of one team on its store `st` (Sec. 5): iterate until an
// iteration changes nothing or some tell finds an empty interval.  Failure is
// checked inside the loop (an infeasible cycle would otherwise keep raising
// bounds); when the loop goes quiet a final scan catches an interval emptied
// by two concurrent tells that each saw a stale opposite bound.
// kTrack = false: the eventless loop of Sec. 5 (every row every iteration).
// kTrack = true: stable rows are skipped.  With full = true every row runs
// in the first iteration (a store nothing is known about); with full = false
// only the rows marked in change buffer 2 do (a fixed point strengthened by a
// few tells, each marked by the caller with mark_changed(.., 2, v)).  Later
// iterations run the rows whose inputs changed in the iteration before.
// Preconditions (published to the team by a barrier): st staged; change
// buffer 0 cleared; buffer 2 cleared except for the caller's marks when
// full = false; fc->fail, evals, bytes == 0.  The caller must not modify *fc
// or the change buffers before the next team barrier after this returns.
// Team-uniform return value; fc->evals / fc->bytes are valid after return
// for the team's thread 0 (for every thread after the next team barrier).
// kGlobal: the table is in global memory; kStream (with kGlobal): its rows
// come in segments through the team's stream *sm, else they are read where
// tb points.  A stream that lost a copy ends the loop with kError.
// kBitSel (global tables): kBitsAny reads the model's layout at run time,
// kBitsNo / kBitsYes compile one sweep (models known to keep no Booleans as
// bits / to keep some).
constexpr int kBitsNo = 0, kBitsYes = 1, kBitsAny = 2;
template <bool kTrack, bool kGlobal = false, bool kStream = false, int kBitSel = kBitsAny,
          bool kSplit = false>
__device__ __forceinline__ int team_fixpoint(const Tab& tb, int2* st, const Team& tm, FixCtrl* fc,
                                             const Track& tk, bool full, int max_iter,
                                             int& iters, Streamer* sm = nullptr) {
  int it = 0;
  constexpr bool kClaim = kGlobal && !kStream;  // sweep_rows claims rows dynamically
  if (kClaim) {  // counter of the first sweep; the barrier publishes it
    if (tm.tid == 0) {
      fc->grab[0] = 0;
      fc->grab[1] = 0;
    }
    team_bar(tm.bar, tm.nthr);
  }
  for (;;) {
    const int cur = it % 3, prv = (it + 2) % 3, nxt = (it + 1) % 3;
    if (kTrack) {
      for (int i = tm.tid; i < tk.W; i += tm.nthr) tk.chg[nxt * tk.W + i] = 0u;
      for (int i = tm.tid; i < tk.WL; i += tm.nthr) tk.dl[nxt * tk.WL + i] = 0u;
    }
    // the next sweep's counter was last used by the previous sweep, which
    // every warp left before the last barrier; this sweep's barrier publishes it
    if (kClaim && tm.tid == 0) fc->grab[(it + 1) & 1] = 0;
    const Sweep w{tb, st,   tk,   cur, tk.chg + prv * tk.W, tk.dl + prv * tk.WL, full || !kTrack,
                  kClaim ? &fc->grab[it & 1] : nullptr};
    Flags f{false, false, 0, 0};
    if (kStream)
      sweep_rows_streamed<kTrack>(w, tm, f, *sm);
    else if (kGlobal && kBitSel != kBitsNo && (kBitSel == kBitsYes || tb.bit0 < tb.n_vars))
      sweep_rows<kTrack, kGlobal, kGlobal>(w, tm, f);  // Booleans kept as bits
    else
      sweep_rows<kTrack, kGlobal, false, kSplit && !kGlobal>(w, tm, f);
    if (kTrack) {  // rows skipped vary: count what ran
      const int ev = __reduce_add_sync(0xffffffffu, f.evals);
      const int by = __reduce_add_sync(0xffffffffu, f.bytes);
      if (tm.lane == 0) {
        atomicAdd(&fc->evals, ev);
        atomicAdd(&fc->bytes, by);
      }
    }
    if (f.fl) st_relaxed(&fc->fail, 1);
    ++it;
    full = false;
    const bool any = team_bar_or(tm.bar, tm.nthr, f.ch || f.fl);
    if (kStream && ld_relaxed(&sm->ctl->err)) {
      iters = it;
      count_sweeps<kTrack>(tb, tm, fc, it);
      return kError;
    }
    if (ld_relaxed(&fc->fail)) {
      iters = it;
      count_sweeps<kTrack>(tb, tm, fc, it);
      return kFailed;
    }
    if (!any) break;
    if (it >= max_iter) {
      iters = it;
      count_sweeps<kTrack>(tb, tm, fc, it);
      return kError;
    }
  }
  count_sweeps<kTrack>(tb, tm, fc, it);
  bool empty = false;
  for (int sl = tm.tid; sl < tb.n_slots; sl += tm.nthr) empty |= slot_empty(ld_dom(st, sl), sl, tb.bit0);
  iters = it;
  return team_bar_or(tm.bar, tm.nthr, empty) ? kFailed : kFixpoint;
}

// Clear change buffers 0 and 2 (before a fixed point); team threads, strided.
__device__ __forceinline__ void track_clear02(const Track& tk, const Team& tm) {
  for (int i = tm.tid; i < tk.W; i += tm.nthr) {
    tk.chg[i] = 0u;
    tk.chg[2 * tk.W + i] = 0u;
  }
  for (int i = tm.tid; i < tk.WL; i += tm.nthr) {
    tk.dl[i] = 0u;
    tk.dl[2 * tk.WL + i] = 0u;
  }
}

// ------------------------------------------------ bulk copy of the table image

// Copy the table image into shared memory with TMA bulk copies issued by
// thread 0 of the CTA; every thread waits (bounded) for completion.  Must be
// called by all threads of the CTA.  `parity` is the mbarrier phase to wait
// for (flip it after each use).  Returns false if the wait gave up; then the
// caller must not read the image.
__device__ __forceinline__ bool load_image(uint8_t* dst, const uint8_t* src, uint32_t bytes,
                                           uint64_t* mbar, uint32_t parity) {
  __syncthreads();  // earlier generic-proxy reads of dst are done
  if (threadIdx.x == 0) {
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
  return __syncthreads_and(ok) != 0;
}

}  // namespace pccp
