// ctx.h -- the library context (internal): scratch arena, streams, events,
// device error word, tuning options and the ragged-launch graph cache.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "host_plan.h"

namespace snt {
inline constexpr int kMaxInject = 64;
// Phase events of one keygen call (snt_ctx_set_timing): on the main stream
// 0 start, 1 after sampling f, 4 after the up-sweep (or per-key R/q
// inversions), 5 after the root, 6 after the down-sweep, 7 after the join,
// 8 after h/encode, 9 after SHA-512; on the auxiliary stream 2 / 3 around the
// R/3 kernel.
inline constexpr int kPhaseEvents = 11;
inline constexpr size_t kMaxB = (size_t)1 << 24;
inline constexpr int kMaxParts = 4;  // pipelined parts of one batch keygen call


// Cached CUDA graph of one ragged launch plan (the list of (P, B) pairs).
struct RaggedGraph {
    std::vector<int> sig;            // P and B of every batch, in call order
    cudaGraphExec_t exec = nullptr;
    size_t table_off = 0, table_bytes = 0;  // device tables inside the arena
};

}  // namespace snt

struct snt_ctx {
    int device = 0;
    size_t budget = 0;
    uint8_t *arena = nullptr;
    int *d_err = nullptr;
    uint64_t *d_inj_idx = nullptr;
    int8_t *d_inj_g = nullptr;
    int n_inj = 0;
    int inj_P = 0;
    cudaStream_t aux = nullptr;   // high priority: the R/3 inversions
    cudaStream_t tree = nullptr;  // high priority: sampling, product tree, h, hash
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_done = nullptr, ev_r3fork = nullptr;
    cudaEvent_t ev_gready = nullptr;       // R/3 batch path: every g final
    cudaStream_t side = nullptr;  // low priority: leaf-pair products s beside the root inversions
    // host-buffer calls that do not wait (snt_batch_keygen_host_async): two
    // staging slots, the copy streams, per slot the events of its pk and sk
    // copies, and the event the copies start from
    cudaStream_t copy[2] = {};
    cudaEvent_t ev_staged[2][2] = {};
    cudaEvent_t ev_kdone = nullptr;
    int stage_next = 0;
    bool copies_pending = false;  // such copies may be in flight (until snt_ctx_sync)
    int async_P = 0;              // parameter set and batch size of the last such call
    size_t async_B = 0;
    cudaEvent_t ev_sfork = nullptr, ev_sready = nullptr;  // fork to / join from the side stream
    uint32_t *d_r3fac[3] = {nullptr, nullptr, nullptr};  // F_3 factors per parameter set
    uint32_t *d_r3screen[3] = {nullptr, nullptr, nullptr};  // small factors' remainder tables
    bool timing = false;
    cudaEvent_t ev_phase[snt::kPhaseEvents] = {};
    int r3_lanes = snt::kDefaultR3Lanes;
    int tree_split = snt::kDefaultTreeSplit;
    int r3_overlap = snt::kDefaultR3Overlap;
    int narrow_seg = snt::kDefaultNarrowSeg;
    int rq_engine = snt::kDefaultRqEngine;
    int mma_tiles = snt::kDefaultMmaTiles;
    int r3_kpt = snt::kDefaultR3Kpt;
    int mma_ksplit = snt::kDefaultMmaKsplit;
    int roots = snt::kDefaultRoots;
    int r3_mode = snt::kDefaultR3Mode;
    int fuse_leaf = 1;  // h from the level-1 inverses (where FuseLeaf<P>::ok)
    int perkey_inv = 1; // per-key path: 1 jump divsteps, 0 one divstep per barrier
    int parts = 1;      // pipelined parts of a batch keygen call (SNT_OPT_PARTS)
    int pdl = 1;        // programmatic dependent launches (SNT_OPT_PDL)
    int r3_roots = 0;   // subtrees of the R/3 forest (SNT_OPT_R3_ROOTS; 0: as the R/q forest)
    cudaStream_t part[snt::kMaxParts - 1] = {};  // streams of parts 1 .. kMaxParts-1
    cudaEvent_t ev_pfork = nullptr, ev_pdone[snt::kMaxParts] = {};
    cudaEvent_t ev_psfork[snt::kMaxParts] = {}, ev_psready[snt::kMaxParts] = {};
    // autotuned options per (parameter set, ceil(log2 B)); lanes == 0: none
    struct Tuned {
        int lanes = 0, split = 0, overlap = 0, engine = 0, tiles = 1, kpt = 1, roots = 1, r3mode = 0;
        int parts = 1, r3roots = 0;
    };
    Tuned tuned[3][25];
    cudaStream_t tune = nullptr;  // stream used while autotuning
    snt::RaggedGraph ragged;      // last ragged plan and its graph
    // ragged launches: per parameter set a main and an R/3 stream and their
    // fork / g-ready / join / done events (created on first use)
    bool rg_ready = false;
    cudaStream_t rg_main[3] = {}, rg_aux[3] = {};
    cudaEvent_t rg_ev[3][5] = {};
};


namespace snt {
inline int pidx(int P) { return P == 653 ? 0 : P == 761 ? 1 : 2; }
inline int bbucket(size_t B) {
    int b = 0;
    while (((size_t)1 << b) < B && b < 24) ++b;
    return b;
}
// Device copy of the F_3 factors of x^P - x - 1 for the R/3 batch path
// (computed on the host on first use; r3batch.cu).
snt_status r3_factors_for(snt_ctx *ctx, int P, R3Factors &out);
// Orders stream st after the copies of snt_batch_keygen_host_async calls
// that may still read their staging slots, before st's work overwrites
// scratch (any call that uses the context's scratch calls it first).
snt_status order_after_copies(snt_ctx *ctx, cudaStream_t st);
snt_status r3_screen_for(snt_ctx *ctx, int P, R3Screen &out);
}  // namespace snt
