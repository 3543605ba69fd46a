// k_propagate.cuh -- the batched propagation kernel (included by pccp.cu).
//
// Persistent CTAs; the packed propagator table is brought into shared memory
// once per CTA by TMA bulk copies (or, when it does not fit beside a store,
// streamed through a ring of per-team buffers every sweep); each team of warps
// pulls stores from a global counter, stages one store (joined with the root
// domains) into shared memory and runs the lock-free fixed-point loop on it
// (Sec. 4-5).
#pragma once

#include "pccp_device.cuh"

namespace pccp {

struct PropArgs {
  const uint8_t* image;
  const int2* root;
  int32_t* lb;
  int32_t* ub;
  int32_t* status;
  int32_t* iters;
  int32_t* work;  // [n_stores][2] {rows evaluated, algorithmic bytes} or null
  int* counter;
  uint32_t image_bytes;
  int n_vars;
  int n_slots;  // store slots per team (variables below bit0, then Boolean words)
  int n_stores;
  int team_size;
  int teams;
  int max_iter;
  int track_words;
  int table_global;   // 1: rows are read from the device image (too big for shared memory)
  int stream_stages;  // table_global: buffers of each team's stream (0: rows read in place)
  int reordered;      // 1: st uses the library's variable order (internal_of after the root)
  uint32_t tlev_bytes;  // table_global, in place: temporal levels staged per CTA (0: none)
  uint32_t off_tlev;    // their offset in the image
  int levels;           // temporal levels: bit 0 staged tables, bit 1 global ones
};

// Per-team scalars of k_propagate (shared memory).
struct PropCtrl {
  int next;
  int pad[3];
  FixCtrl fc;
};

// Instantiated for 1024-thread CTAs (one per SM) and for CTAs of up to 512
// threads with three resident per SM (registers capped for 48 warps/SM);
// kGlobal: the table is read from global memory (1024-thread variant only),
// in place or, with kStream (stream_stages > 0), streamed.
template <int kMaxThreads, int kMinBlocks, bool kTrack, bool kGlobal, bool kStream>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks) k_propagate(PropArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  // shared memory: [table image | kGlobal: one stream region per team, or
  //                 the temporal levels, or none]
  //                [mbarrier 16 B][PropCtrl x teams][change words x teams][stores]
  const size_t stream_region = stream_bytes(a.stream_stages);
  const uint32_t tl_bytes = kGlobal && !kStream ? a.tlev_bytes : 0u;
  const size_t img_bytes = kGlobal ? stream_region * a.teams + tl_bytes : a.image_bytes;
  uint8_t* img = smem;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + img_bytes);
  PropCtrl* ctrl_base = reinterpret_cast<PropCtrl*>(smem + img_bytes + 16);
  const int tw16 = (a.track_words + 3) & ~3;  // words, 16-byte multiple
  uint32_t* track_base =
      reinterpret_cast<uint32_t*>(smem + img_bytes + 16 + sizeof(PropCtrl) * a.teams);
  int2* st_base = reinterpret_cast<int2*>(track_base + static_cast<size_t>(tw16) * a.teams);

  bool ok = true;
  if (!kGlobal) {
    if (threadIdx.x == 0) mbar_init(mbar, 1);
    ok = load_image(img, a.image, a.image_bytes, mbar, 0);
  } else if (tl_bytes != 0u) {  // 16-byte multiples at 16-byte aligned offsets
    const int4* src = reinterpret_cast<const int4*>(a.image + a.off_tlev);
    int4* dst = reinterpret_cast<int4*>(smem);
    const uint32_t n16 = a.tlev_bytes / 16u;
    for (uint32_t i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
  }

  const int team_id = threadIdx.x / a.team_size;
  Team tm;
  tm.tid = threadIdx.x - team_id * a.team_size;
  tm.nthr = a.team_size;
  tm.bar = 1 + team_id;
  tm.lane = threadIdx.x & 31;
  tm.warp = tm.tid >> 5;
  tm.nwarps = a.team_size >> 5;
  PropCtrl* ctrl = ctrl_base + team_id;
  int2* st = st_base + static_cast<size_t>(team_id) * a.n_slots;
  Tab tb = make_tab(kGlobal ? a.image : img, a.levels & (kGlobal ? 2 : 1));
  if (kGlobal) {  // the levels from shared memory, or the rows one thread each
    if (tl_bytes != 0u)
      tab_levels_at(tb, smem);
    else
      tb.n_tlev = 0;
  }
  const Track tk = make_track(track_base + static_cast<size_t>(tw16) * team_id, tb.n_vars,
                              tb.n_lin + tb.n_lin_long);
  const int nv = a.n_vars;
  // the library's index of each of the caller's variables (after the root)
  const int32_t* internal_of = reinterpret_cast<const int32_t*>(a.root + nv);
  Streamer stream;
  if (kStream)  // published by the barrier at the top of the store loop
    stream = stream_open(smem + stream_region * team_id, a.stream_stages, tb, a.image, tm, 0u);

  for (;;) {
    if (tm.tid == 0) ctrl->next = atomicAdd(a.counter, 1);
    team_bar(tm.bar, tm.nthr);
    const int s = ctrl->next;
    if (s >= a.n_stores) break;
    if (!ok) {  // table never arrived: report the stores this team takes
      if (tm.tid == 0) {
        a.status[s] = kError;
        if (a.iters) a.iters[s] = 0;
        if (a.work) {
          a.work[2 * static_cast<size_t>(s)] = 0;
          a.work[2 * static_cast<size_t>(s) + 1] = 0;
        }
      }
      continue;
    }
    // stores are in the caller's variable order, st in the library's
    int32_t* lbs = a.lb + static_cast<size_t>(s) * nv;
    int32_t* ubs = a.ub + static_cast<size_t>(s) * nv;
    bool empty = false;
    const int b0 = tb.bit0;
    for (int x = tm.tid; x < nv; x += tm.nthr) {
      const int v = a.reordered ? __ldg(internal_of + x) : x;
      if (v >= b0) continue;  // a Boolean kept as a bit: staged below
      const int2 r = __ldg(a.root + v);
      const int l = max(lbs[x], r.x), u = min(ubs[x], r.y);
      st[v] = make_int2(l, u);
      empty |= l > u;
    }
    // Booleans kept as bits: a warp per slot of 32, lane j the library's
    // variable bit0 + 32 slot + j; the slot's two words come from ballots (an
    // empty input interval leaves its bit empty: lower set, upper clear)
    for (int wi = tm.warp; b0 + wi < tb.n_slots; wi += tm.nwarps) {
      const int v = b0 + 32 * wi + tm.lane;
      bool lbit = false, ubit = true;
      if (v < nv) {
        const int x = __ldg(internal_of + nv + v);  // the caller's index (user_of)
        const int2 r = __ldg(a.root + v);
        const int l = max(lbs[x], r.x), u = min(ubs[x], r.y);
        lbit = l > u || l >= 1;
        ubit = l <= u && u >= 1;
        empty |= l > u;
      }
      const uint32_t lw = __ballot_sync(0xffffffffu, lbit);
      const uint32_t uw = __ballot_sync(0xffffffffu, ubit);
      if (tm.lane == 0) st[b0 + wi] = make_int2(static_cast<int>(lw), static_cast<int>(uw));
    }
    if (kTrack) track_clear02(tk, tm);
    if (tm.tid == 0) {
      ctrl->fc.fail = 0;
      ctrl->fc.evals = 0;
      ctrl->fc.bytes = 0;
    }
    const bool any_empty = team_bar_or(tm.bar, tm.nthr, empty);
    int status = kFailed, it = 0;
    if (!any_empty)
      status = team_fixpoint<kTrack, kGlobal, kStream>(tb, st, tm, &ctrl->fc, tk, true,
                                                       a.max_iter, it, &stream);
    for (int x = tm.tid; x < nv; x += tm.nthr) {
      const int2 D = var_dom_plain(st, b0, a.reordered ? __ldg(internal_of + x) : x);
      lbs[x] = D.x;
      ubs[x] = D.y;
    }
    if (tm.tid == 0) {
      a.status[s] = status;
      if (a.iters) a.iters[s] = it;
      if (a.work) {
        a.work[2 * static_cast<size_t>(s)] = ctrl->fc.evals;
        a.work[2 * static_cast<size_t>(s) + 1] = ctrl->fc.bytes;
      }
    }
  }
  // every thread passed the barrier after its last segment: the copies in
  // flight are the prefetched ones
  if (kStream) stream_close(stream);
}

}  // namespace pccp
