// ragged.cu -- many key-generation batches of different sizes and parameter
// sets in one graph launch (snt_batch_keygen_ragged).
//
// Every batch is its own instance of Algorithm 1 (its own Montgomery product
// tree, Sec. 2.2, with its own root inversion), so its bytes are exactly
// those of snt_batch_keygen on that batch alone.  The batches of one
// parameter set form a forest that is processed level by level: one launch
// per tree level covers the nodes of every batch at that level (CTA -> batch
// by a binary search over per-level prefix sums), one launch inverts every
// batch's root, and the per-key kernels (sampling, h and Rq_encode, SHA-512)
// run once over all keys of the parameter set, looking up each key's batch in
// a device table.  The inverses of g in R/3 are either per key (divsteps, on
// a second stream beside the R/q forest, redrawn keys fixed up at the end) or
// batched as in Sec. 3.1.1: every g tested invertible by its remainders modulo
// the F_3 factors of x^p - x - 1 (and redrawn until it is), then one R/3
// forest with the same shape as the R/q forest.  The three parameter sets run
// on their own pairs of streams, side by side.  Each parameter set takes the
// layouts the autotuner chose for (p, the bucket of its largest batch) on this
// context, else the context's options.  The sequence of launches for a plan
// (the list of (p, B) pairs and the layouts) is captured once into a CUDA graph
// and replayed; per-call data (seeds, key indices, output pointers) lives in
// device tables uploaded before each replay.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "pdl.cuh"

using namespace snt;

namespace {

#define SNT_CUDA_R(call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return set_error(SNT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));          \
    } while (0)

// Host plan of the batches of one parameter set.
struct Group {
    int P = 0;
    ParamInfo pi;
    std::vector<int> batch;               // indices into the call's arrays
    int nkeys = 0, L = 0;                 // keys, number of levels above the leaves
    std::vector<std::vector<int>> pre;    // [level][batch + 1] node prefix sums
    std::vector<int> lev_off;             // first node of each level (nodes)
    std::vector<int> root_row;            // node row of each batch's root
    size_t nodes = 0;                     // node rows in the forest
    // arena offsets (bytes): tree nodes, g rows, resampling list (count and
    // keys, then final g rows) of the deferred R/3 kernel, R/3 forest nodes
    size_t off_nodes = 0, off_g = 0, off_fix = 0, off_gfix = 0, off_nodes3 = 0;
    // kernel layouts of this parameter set
    int lanes = 4, split = 8, tiles = 1, kpt = 1, ksplit = 4;
    // r3batch: R/3 inverses by the batch forest; r3first: on the first draws
    // (invertibility from each batch's root, a failed batch redone per key)
    bool mma = true, ntt = false, wide = false, r3batch = false, r3first = false, fuse = false;
    size_t off_r3ok = 0;  // one root flag per batch (r3first)
    R3Factors fac;
    R3Screen scr;  // the small factors' remainder tables (mode 2)
    // table offsets (bytes, from the start of the uploaded table block)
    size_t t_desc = 0, t_pre = 0, t_root = 0;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Level structure of the batches of one parameter set.  min_levels = 1 (the
// fused leaf level) gives a one-key batch a level-1 node too (its leaf moved
// up unchanged), so that every batch's keys sit under level-1 nodes.  A
// batch's root is its node on the last level where it has one.
void plan_group(Group &g, const size_t *B, int min_levels) {
    const int nb = (int)g.batch.size();
    std::vector<int> n(nb), next(nb);
    for (int i = 0; i < nb; ++i) {
        n[i] = (int)B[g.batch[i]];
        g.nkeys += n[i];
    }
    g.root_row.assign(nb, 0);
    g.lev_off.clear();
    g.pre.clear();
    size_t off = 0;
    for (int l = 0;; ++l) {
        std::vector<int> pre(nb + 1, 0);
        for (int i = 0; i < nb; ++i) pre[i + 1] = pre[i] + n[i];
        g.pre.push_back(pre);
        g.lev_off.push_back((int)off);
        bool more = false;
        for (int i = 0; i < nb; ++i) {
            next[i] = n[i] > 1 ? (n[i] + 1) / 2 : (n[i] == 1 && l + 1 <= min_levels ? 1 : 0);
            if (n[i] == 1 && next[i] == 0) g.root_row[i] = (int)off + pre[i];
            more = more || next[i] > 0;
        }
        off += pre[nb];
        n = next;
        if (!more) break;
        g.L = l + 1;
    }
    g.nodes = off;
}

template <int P>
snt_status launch_group(snt_ctx *ctx, const Group &g, uint8_t *tables, cudaStream_t st,
                        cudaStream_t aux, cudaEvent_t ev_fork, cudaEvent_t ev_gready,
                        cudaEvent_t ev_join) {
    const ParamInfo &pi = g.pi;
    const int nb = (int)g.batch.size();
    int16_t *nodes = reinterpret_cast<int16_t *>(ctx->arena + g.off_nodes);
    int16_t *nodes3 = reinterpret_cast<int16_t *>(ctx->arena + g.off_nodes3);
    int8_t *gbuf = reinterpret_cast<int8_t *>(ctx->arena + g.off_g);
    int *fix_count = reinterpret_cast<int *>(ctx->arena + g.off_fix);
    int *fix_keys = fix_count + 1;
    int *fix_slot = fix_keys + g.nkeys;  // by key: the R/3 screen's slot, or -1
    int8_t *gfix = reinterpret_cast<int8_t *>(ctx->arena + g.off_gfix);
    int *r3ok = reinterpret_cast<int *>(ctx->arena + g.off_r3ok);
    KeyMap km;
    std::memset(&km, 0, sizeof(km));
    km.tab = reinterpret_cast<const BatchDesc *>(tables + g.t_desc);
    km.nb = nb;
    const int *pre = reinterpret_cast<const int *>(tables + g.t_pre);  // [level][nb + 1]
    const int *roots = reinterpret_cast<const int *>(tables + g.t_root);
    const int sb = pi.small_bytes;
    auto lmap = [&](int l) {
        LevelMap lm;
        lm.pre_in = pre + (size_t)(l - 1) * (nb + 1);
        lm.pre_out = pre + (size_t)l * (nb + 1);
        lm.nb = nb;
        lm.n_in = 0;
        return lm;
    };
    // g's first draw with f; the R/3 work runs on the auxiliary stream beside
    // the R/q forest and is joined at the end
    // (r3first: g's first draws also go to the R/3 leaves, as int16)
    // the test hook's injected first draws (snt_debug_inject_g): by key index
    const int n_inj = (ctx->inj_P == P) ? ctx->n_inj : 0;
    SNT_CUDA_R(launch_sample_f<P>(km, g.nkeys, nodes, pi.sk_bytes, 2 * sb + pi.pk_bytes, st, gbuf,
                                  ctx->d_inj_idx, ctx->d_inj_g, n_inj, fix_count,
                                  g.r3first ? nodes3 : nullptr));
    SNT_CUDA_R(cudaEventRecord(ev_fork, st));
    SNT_CUDA_R(cudaStreamWaitEvent(aux, ev_fork, 0));
    if (g.r3batch) {
        // Sec. 3.1.1: isInvertible (remainders modulo the F_3 factors) with
        // redraws, final g into the R/3 leaves, then Montgomery's trick in R/3
        // over the same forest shape, one jump-divstep root per batch; or
        // (r3first) the forest on the first draws, a batch whose root does
        // not invert (some g in it is a zero divisor) redone per key below
        if (!g.r3first) {
            SNT_CUDA_R(launch_r3_check<P>(km, g.nkeys, gbuf, nodes3, g.fac, ctx->d_err, aux));
            SNT_CUDA_R(cudaEventRecord(ev_gready, aux));
        } else if (g.scr.n > 0) {  // first draws screened against the small factors
            SNT_CUDA_R(launch_r3_screen<P>(km, g.nkeys, gbuf, nodes3, g.scr, gfix, fix_count,
                                           fix_keys, fix_slot, ctx->d_err, aux));
        }
        for (int l = 1; l <= g.L; ++l)
            SNT_CUDA_R(launch_tree_up_mma3<P>(nodes3 + (size_t)g.lev_off[l - 1] * pi.pad, lmap(l),
                                              g.pre[l][nb], nodes3 + (size_t)g.lev_off[l] * pi.pad,
                                              aux, g.ksplit));
        SNT_CUDA_R(launch_r3_inv_jump<P>(nb, nodes3, pi.pad, nodes3, pi.pad,
                                         g.r3first ? r3ok : nullptr,
                                         g.r3first ? nullptr : ctx->d_err, ERR_ROOT, aux, roots));
        for (int l = g.L; l >= 1; --l)
            SNT_CUDA_R(launch_tree_down_mma3<P>(nodes3 + (size_t)g.lev_off[l] * pi.pad, lmap(l),
                                                g.pre[l][nb],
                                                nodes3 + (size_t)g.lev_off[l - 1] * pi.pad, aux,
                                                g.ksplit));
        SNT_CUDA_R(launch_r3_encode_v<P>(km, g.nkeys, nodes3, pi.sk_bytes, sb, aux,
                                         g.r3first ? r3ok : nullptr, 0));
        if (g.r3first)  // batches whose root did not invert: per key, with redraws
            SNT_CUDA_R(launch_r3_keygen<P>(km, g.nkeys, gbuf, pi.sk_bytes, sb, ctx->d_inj_idx,
                                           ctx->d_inj_g, n_inj, ctx->d_err, aux, g.lanes, g.kpt,
                                           gfix, fix_count, fix_keys, r3ok, 0,
                                           g.scr.n > 0 ? fix_slot : nullptr));
    } else {
        SNT_CUDA_R(launch_r3_keygen<P>(km, g.nkeys, gbuf, pi.sk_bytes, sb, ctx->d_inj_idx,
                                       ctx->d_inj_g, n_inj, ctx->d_err, aux, g.lanes, g.kpt, gfix,
                                       fix_count, fix_keys));
    }
    SNT_CUDA_R(cudaEventRecord(ev_join, aux));
    for (int l = 1; l <= g.L; ++l) {
        const int n_out = g.pre[l][nb];
        if (g.ntt && l > 1)
            SNT_CUDA_R(launch_tree_up_ntt<P>(nodes + (size_t)g.lev_off[l - 1] * pi.pad, lmap(l),
                                             n_out, nodes + (size_t)g.lev_off[l] * pi.pad, st));
        else if (g.mma)
            SNT_CUDA_R(launch_tree_up_mma<P>(nodes + (size_t)g.lev_off[l - 1] * pi.pad, lmap(l),
                                             n_out, nodes + (size_t)g.lev_off[l] * pi.pad, st,
                                             g.tiles, l == 1, g.ksplit, g.wide));
        else
            SNT_CUDA_R(launch_tree_up<P>(nodes + (size_t)g.lev_off[l - 1] * pi.pad, lmap(l), n_out,
                                         nodes + (size_t)g.lev_off[l] * pi.pad, st, g.split));
    }
    SNT_CUDA_R(launch_rq_inv_jump<P>(nb, nodes, pi.pad, nodes, pi.pad, nullptr, ctx->d_err,
                                     ERR_ROOT, st, roots));
    for (int l = g.L; l >= (g.fuse ? 2 : 1); --l) {
        const int n_par = g.pre[l][nb];
        if (g.ntt && l > 1)
            SNT_CUDA_R(launch_tree_down_ntt<P>(nodes + (size_t)g.lev_off[l] * pi.pad, lmap(l),
                                               n_par, nodes + (size_t)g.lev_off[l - 1] * pi.pad, st));
        else if (g.mma)
            SNT_CUDA_R(launch_tree_down_mma<P>(nodes + (size_t)g.lev_off[l] * pi.pad, lmap(l),
                                               n_par, nodes + (size_t)g.lev_off[l - 1] * pi.pad,
                                               st, g.tiles, l == 1, g.ksplit, g.wide));
        else
            SNT_CUDA_R(launch_tree_down<P>(nodes + (size_t)g.lev_off[l] * pi.pad, lmap(l), n_par,
                                           nodes + (size_t)g.lev_off[l - 1] * pi.pad, st, g.split));
    }
    if (g.r3batch && !g.r3first)  // h needs the final g
        SNT_CUDA_R(cudaStreamWaitEvent(st, ev_gready, 0));
    if (g.fuse)
        SNT_CUDA_R(launch_finalize_pair<P>(km, g.pre[1][nb], gbuf, nodes,
                                           nodes + (size_t)g.lev_off[1] * pi.pad, lmap(1),
                                           pi.pk_bytes, pi.sk_bytes, 2 * sb, pi.sched, st,
                                           nullptr));
    else
        SNT_CUDA_R(launch_finalize<P>(km, g.nkeys, gbuf, nodes, pi.pk_bytes, pi.sk_bytes, 2 * sb,
                                      pi.sched, st, g.mma));
    SNT_CUDA_R(launch_sha512_pk(km, g.nkeys, pi.pk_bytes, pi.sk_bytes, 3 * sb + pi.pk_bytes, st));
    SNT_CUDA_R(cudaStreamWaitEvent(st, ev_join, 0));
    if (!g.r3batch || g.r3first)  // keys whose g a per-key R/3 kernel redrew: h, pk, hash again
        SNT_CUDA_R(launch_fixup<P>(km, fix_count, fix_keys, gfix,
                                   g.fuse ? nodes + (size_t)g.lev_off[1] * pi.pad : nodes,
                                   pi.pk_bytes, pi.sk_bytes, 2 * sb, 3 * sb + pi.pk_bytes, pi.sched,
                                   st, g.fuse ? nodes : nullptr, lmap(1), fixup_grid(g.nkeys), g.nkeys));
    return SNT_OK;
}

// Streams and events of the three parameter sets' branches (created on the
// first ragged call, kept for the context's life).
snt_status ensure_ragged_streams(snt_ctx *ctx) {
    if (ctx->rg_ready) return SNT_OK;
    int lo = 0, hi = 0;
    SNT_CUDA_R(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    for (int j = 0; j < 3; ++j) {
        SNT_CUDA_R(cudaStreamCreateWithPriority(&ctx->rg_main[j], cudaStreamNonBlocking, hi));
        SNT_CUDA_R(cudaStreamCreateWithPriority(&ctx->rg_aux[j], cudaStreamNonBlocking, hi));
        for (int e = 0; e < 5; ++e)
            SNT_CUDA_R(cudaEventCreateWithFlags(&ctx->rg_ev[j][e], cudaEventDisableTiming));
    }
    ctx->rg_ready = true;
    return SNT_OK;
}

}  // namespace

extern "C" snt_status snt_batch_keygen_ragged(snt_ctx *ctx, size_t n_batches, const int *P,
                                              const size_t *B, const uint64_t *seeds,
                                              const uint64_t *first_idx, uint8_t *const *pk_dev,
                                              uint8_t *const *sk_dev, snt_stream stream) {
    if (!ctx) return set_error(SNT_EINVAL, "null context");
    if (n_batches == 0 || n_batches > 65536)
        return set_error(SNT_EINVAL, "batch count %zu outside [1, 65536]", n_batches);
    if (!P || !B || !seeds || !first_idx || !pk_dev || !sk_dev)
        return set_error(SNT_EINVAL, "null argument array");
    Group groups[3];
    const int Ps[3] = {653, 761, 857};
    size_t total = 0;
    for (size_t i = 0; i < n_batches; ++i) {
        int gi = -1;
        for (int j = 0; j < 3; ++j)
            if (P[i] == Ps[j]) gi = j;
        if (gi < 0) return set_error(SNT_EINVAL, "batch %zu: unknown parameter set %d", i, P[i]);
        if (B[i] == 0 || B[i] > kMaxB) return set_error(SNT_EINVAL, "batch %zu: size %zu", i, B[i]);
        if (!pk_dev[i] || !sk_dev[i]) return set_error(SNT_EINVAL, "batch %zu: null output", i);
        total += B[i];
        groups[gi].batch.push_back((int)i);
    }
    if (total > kMaxB) return set_error(SNT_EINVAL, "%zu keys in one call (max %zu)", total, kMaxB);

    // plan: arena layout and device tables
    size_t arena_off = 0, tbytes = 0;
    for (int j = 0; j < 3; ++j) {
        Group &g = groups[j];
        if (g.batch.empty()) continue;
        g.P = Ps[j];
        param_info(g.P, g.pi);
        // layouts: the autotuner's choice for (p, the largest batch's bucket)
        // if it ran on this context, else the context's options
        size_t bmax = 0;
        for (int bi : g.batch) bmax = std::max(bmax, B[bi]);
        const snt_ctx::Tuned &tu = ctx->tuned[pidx(g.P)][bbucket(bmax)];
        g.lanes = ctx->r3_lanes; g.split = ctx->tree_split; g.tiles = ctx->mma_tiles;
        g.kpt = ctx->r3_kpt; g.mma = ctx->rq_engine != 0; g.ntt = ctx->rq_engine == 2;
        g.wide = ctx->rq_engine == 3;
        g.r3batch = ctx->r3_mode != 0;
        g.r3first = ctx->r3_mode == 2;
        g.ksplit = ctx->mma_ksplit;
        if (tu.lanes) {
            g.lanes = tu.lanes; g.split = tu.split; g.tiles = tu.tiles; g.kpt = tu.kpt;
            g.mma = tu.engine != 0; g.ntt = tu.engine == 2; g.wide = tu.engine == 3;
            g.r3batch = tu.r3mode != 0;
            g.r3first = tu.r3mode == 2;
        }
        // h from the level-1 inverses (the down-sweep's leaf level folded
        // into h, as in the single-batch call) needs the tensor-core h kernel
        const bool fuse_ok = g.P == 653 ? FuseLeaf<653>::ok : g.P == 761 ? FuseLeaf<761>::ok
                                                                         : FuseLeaf<857>::ok;
        g.fuse = g.mma && ctx->fuse_leaf && fuse_ok;
        plan_group(g, B, g.fuse ? 1 : 0);
        g.off_nodes = arena_off;
        arena_off += align_up(g.nodes * g.pi.pad * sizeof(int16_t), 256);
        g.off_g = arena_off;
        arena_off += align_up((size_t)g.nkeys * g.pi.pad, 256);
        g.off_fix = arena_off;
        arena_off += align_up(sizeof(int) * (1 + 2 * (size_t)g.nkeys), 256);
        g.off_gfix = arena_off;
        arena_off += align_up((size_t)g.nkeys * g.pi.pad, 256);
        if (g.r3batch) {
            if (!g.r3first) {
                const snt_status sf = r3_factors_for(ctx, g.P, g.fac);
                if (sf != SNT_OK) return sf;
            } else {
                const snt_status ss = r3_screen_for(ctx, g.P, g.scr);
                if (ss != SNT_OK) return ss;
            }
            g.off_nodes3 = arena_off;
            arena_off += align_up(g.nodes * g.pi.pad * sizeof(int16_t), 256);
            g.off_r3ok = arena_off;
            arena_off += align_up(g.batch.size() * sizeof(int), 256);
        }
        const size_t nb = g.batch.size();
        g.t_desc = tbytes;
        tbytes += align_up(nb * sizeof(BatchDesc), 16);
        g.t_pre = tbytes;
        tbytes += align_up((size_t)(g.L + 1) * (nb + 1) * sizeof(int), 16);
        g.t_root = tbytes;
        tbytes += align_up(nb * sizeof(int), 16);
    }
    const size_t table_off = align_up(arena_off, 256);
    if (table_off + tbytes > ctx->budget)
        return set_error(SNT_ENOMEM, "ragged launch needs %zu scratch bytes, budget %zu",
                         table_off + tbytes, ctx->budget);
    std::vector<uint8_t> host(tbytes, 0);
    for (int j = 0; j < 3; ++j) {
        const Group &g = groups[j];
        if (g.batch.empty()) continue;
        const int nb = (int)g.batch.size();
        BatchDesc *d = reinterpret_cast<BatchDesc *>(host.data() + g.t_desc);
        int key_base = 0;
        for (int i = 0; i < nb; ++i) {
            const int bi = g.batch[i];
            d[i].seed = seeds[bi];
            d[i].first = first_idx[bi];
            d[i].key_base = key_base;
            d[i].nkeys = (int)B[bi];
            d[i].pk = pk_dev[bi];
            d[i].sk = sk_dev[bi];
            key_base += (int)B[bi];
        }
        int *pre = reinterpret_cast<int *>(host.data() + g.t_pre);
        for (int l = 0; l <= g.L; ++l)
            for (int i = 0; i <= nb; ++i) pre[(size_t)l * (nb + 1) + i] = g.pre[l][i];
        int *roots = reinterpret_cast<int *>(host.data() + g.t_root);
        for (int i = 0; i < nb; ++i) roots[i] = g.root_row[i];
    }

    DeviceGuard dg(ctx->device);
    if (!dg.ok) return set_error(SNT_ECUDA, "cannot select device %d", ctx->device);
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *tables = ctx->arena + table_off;
    {
        const snt_status so = order_after_copies(ctx, caller);
        if (so != SNT_OK) return so;
    }
    // per-call data first (pageable source: staged before the call returns)
    SNT_CUDA_R(cudaMemcpyAsync(tables, host.data(), tbytes, cudaMemcpyHostToDevice, caller));

    std::vector<int> sig;
    sig.reserve(2 * n_batches);
    for (size_t i = 0; i < n_batches; ++i) {
        sig.push_back(P[i]);
        sig.push_back((int)B[i]);
    }
    RaggedGraph &rg = ctx->ragged;
    // the cached graph holds the kernel layouts: they are part of its key
    for (int j = 0; j < 3; ++j) {
        const Group &g = groups[j];
        if (g.batch.empty()) continue;
        sig.push_back(g.lanes);
        sig.push_back(g.split);
        sig.push_back(g.mma ? g.tiles : 0);
        sig.push_back(g.ntt ? 1 : g.wide ? 2 : 0);
        sig.push_back(g.kpt);
        sig.push_back(g.ksplit);
        sig.push_back(g.r3batch ? (g.r3first ? 2 : 1) : 0);
        sig.push_back(g.fuse ? 1 : 0);
        sig.push_back(ctx->inj_P == g.P ? ctx->n_inj : 0);
    }
    sig.push_back(ctx->pdl);
    if (!(rg.exec && rg.sig == sig && rg.table_off == table_off)) {
        if (rg.exec) cudaGraphExecDestroy(rg.exec);
        rg.exec = nullptr;
        rg.sig.clear();
        const snt_status ss = ensure_ragged_streams(ctx);
        if (ss != SNT_OK) return ss;
        const PdlScope pdl_scope(ctx->pdl != 0);
        // capture from the tree stream: each parameter set forks onto its
        // own pair of streams (its R/3 work onto the second) and joins back
        SNT_CUDA_R(cudaStreamBeginCapture(ctx->tree, cudaStreamCaptureModeThreadLocal));
        snt_status s = SNT_OK;
        cudaError_t ef = cudaEventRecord(ctx->ev_fork, ctx->tree);
        for (int j = 0; j < 3 && s == SNT_OK && ef == cudaSuccess; ++j) {
            const Group &g = groups[j];
            if (g.batch.empty()) continue;
            cudaStream_t gs = ctx->rg_main[j], ga = ctx->rg_aux[j];
            cudaEvent_t *ev = ctx->rg_ev[j];
            ef = cudaStreamWaitEvent(gs, ctx->ev_fork, 0);
            if (ef != cudaSuccess) break;
            switch (g.P) {
                case 653: s = launch_group<653>(ctx, g, tables, gs, ga, ev[0], ev[1], ev[2]); break;
                case 761: s = launch_group<761>(ctx, g, tables, gs, ga, ev[0], ev[1], ev[2]); break;
                default: s = launch_group<857>(ctx, g, tables, gs, ga, ev[0], ev[1], ev[2]); break;
            }
            if (s != SNT_OK) break;
            ef = cudaEventRecord(ev[3], gs);
            if (ef == cudaSuccess) ef = cudaStreamWaitEvent(ctx->tree, ev[3], 0);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(ctx->tree, &graph);
        if (s != SNT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (ef != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return set_error(SNT_ECUDA, "graph capture fork/join: %s", cudaGetErrorString(ef));
        }
        if (ec != cudaSuccess) return set_error(SNT_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&rg.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            rg.exec = nullptr;
            return set_error(SNT_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
        }
        rg.sig = sig;
        rg.table_off = table_off;
        rg.table_bytes = tbytes;
    }
    SNT_CUDA_R(cudaEventRecord(ctx->ev_done, caller));
    SNT_CUDA_R(cudaStreamWaitEvent(ctx->tree, ctx->ev_done, 0));
    SNT_CUDA_R(cudaGraphLaunch(rg.exec, ctx->tree));
    SNT_CUDA_R(cudaEventRecord(ctx->ev_done, ctx->tree));
    SNT_CUDA_R(cudaStreamWaitEvent(caller, ctx->ev_done, 0));
    return SNT_OK;
}
