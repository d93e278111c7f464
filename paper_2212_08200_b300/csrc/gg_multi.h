// gg_multi.h -- the slot engine shared by gg_sssp_multi and the query server.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gg_common.cuh"

namespace gg {

enum : uint32_t { kSlotFree = 0, kSlotRunning = 1, kSlotDone = 2 };

// One query in flight: a graph, a source, the caller's distance array and the
// slot's two dedup bitmaps (word offsets into the engine's bitmap pool).
struct MultiSlot {
  const uint32_t* ro;
  const void* edges;
  uint32_t* dist;
  uint32_t n;
  uint32_t packed, wbits;
  uint32_t src;
  uint32_t bm_off[3];     // near bitmaps (by superstep parity) and the far-pile bitmap
  uint32_t state;
  uint32_t ticket;        // written to the done flag when the query converges
  uint32_t status;        // DS_* bits of this query
  uint32_t supersteps;    // supersteps the query took part in
  // near-far buckets of this query (delta == 0xFFFFFFFF: plain frontier loop)
  uint32_t delta, t_cur, t_prev;
  uint32_t far_off[2];    // its two far piles in the far pool (ping-pong across splits)
  uint32_t far_cnt[2];
  uint32_t fpp;           // current pile
  uint32_t far_min;
  uint32_t split;         // 1: this superstep splits the slot's far pile
};

constexpr int kMaxSplitSlots = 1024;

struct MultiCtl {
  unsigned long long cnt[2];   // (count << 32) | edges of the union frontier, by parity
  uint32_t iter;
  uint32_t done_ctas;
  uint32_t running;            // union frontier non-empty or a split pending
  uint32_t budget_left;        // supersteps this graph launch may still run
  unsigned long long supersteps_run;
  uint32_t nsplit;             // slots splitting in the current superstep
  uint32_t split_total;        // their far entries
  uint32_t split_slot[kMaxSplitSlots];
  uint32_t split_pref[kMaxSplitSlots + 1];
};

struct MultiBufs {
  uint32_t* fv[2];
  uint32_t* fr[2];
  uint32_t* fs[2];
  uint32_t* fq[2];             // slot of each union-frontier entry
  MultiSlot* slots;
  uint32_t* slot_cnt;          // entries each slot appended to the next frontier
  uint32_t* bm_pool;
  uint32_t* far_pool;
  MultiCtl* ctl;
  uint32_t* done_flags;        // device view of host-mapped words (server) or NULL
  uint32_t* done_status;       // device view of host-mapped words (server) or NULL
  uint32_t nslots;
};

struct MultiEngine {
  uint32_t max_slots = 0;
  uint64_t cap_vertices = 0;   // union frontier capacity
  uint64_t cap_words = 0;      // bitmap pool words
  uint64_t cap_far = 0;        // far pool entries
  void* block = nullptr;
  size_t bytes = 0;
  MultiBufs b{};
  uint32_t* starting = nullptr;      // device list of slots being seeded
  MultiSlot* h_slots = nullptr;      // pinned host copy of the slot table
  uint32_t* h_start = nullptr;       // pinned
  MultiCtl* h_ctl = nullptr;         // pinned
  uint32_t* h_done = nullptr;        // mapped pinned (server)
  uint32_t* h_done_status = nullptr; // mapped pinned (server)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int grid = 0;
};

gg_status multi_engine_init(MultiEngine* e, uint32_t max_slots, uint64_t max_vertices, uint64_t max_bitmap_words,
                            uint64_t max_far, bool mapped_flags);
// fills the near-far fields of a slot descriptor (delta 0xFFFFFFFF = none)
void multi_slot_buckets(MultiSlot& s, uint32_t delta, uint32_t far0, uint32_t far1);
void multi_engine_free(MultiEngine* e);
// zero the union frontier and the counters (no query in flight)
gg_status multi_engine_reset(MultiEngine* e, cudaStream_t s);
// upload the host slot descriptors of `slots` (already filled in e->h_slots),
// set their distances to INF, clear their bitmaps and seed their sources
gg_status multi_engine_start(MultiEngine* e, const uint32_t* slots, uint32_t count, cudaStream_t s);
// run supersteps until the union frontier empties or `budget` supersteps ran
gg_status multi_engine_run(MultiEngine* e, uint32_t budget, cudaStream_t s);

}  // namespace gg
