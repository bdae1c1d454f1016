// ragged.cu -- many key-generation batches of different sizes and parameter
// sets in one graph launch (snt_batch_keygen_ragged).
//
// Every batch is its own instance of Algorithm 1 (its own Montgomery product
// tree, Sec. 2.2, with its own root inversion), so its bytes are exactly
// those of snt_batch_keygen on that batch alone.  The batches of one
// parameter set form a forest that is processed level by level: one launch
// per tree level covers the nodes of every batch at that level (CTA -> batch
// by a binary search over per-level prefix sums), one launch inverts every
// batch's root, and the per-key kernels (sampling, R/3 inversion, h and
// Rq_encode, SHA-512) run once over all keys of the parameter set, looking up
// each key's batch in a device table.  The sequence of launches for a plan
// (the list of (p, B) pairs) is captured once into a CUDA graph and replayed;
// per-call data (seeds, key indices, output pointers) lives in device tables
// uploaded before each replay.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.h"

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
    // keys, then final g rows) of the deferred R/3 kernel
    size_t off_nodes = 0, off_g = 0, off_fix = 0, off_gfix = 0;
    // table offsets (bytes, from the start of the uploaded table block)
    size_t t_desc = 0, t_pre = 0, t_root = 0;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void plan_group(Group &g, const size_t *B) {
    const int nb = (int)g.batch.size();
    std::vector<int> n(nb);
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
        for (int i = 0; i < nb; ++i)
            if (n[i] == 1 && (l == 0 || g.pre[l - 1][i + 1] - g.pre[l - 1][i] > 1))
                g.root_row[i] = (int)off + pre[i];  // the level where batch i reaches one node
        off += pre[nb];
        bool more = false;
        for (int i = 0; i < nb; ++i) {
            n[i] = (n[i] > 1) ? (n[i] + 1) / 2 : 0;
            more = more || n[i] > 0;
        }
        if (!more) break;
        g.L = l + 1;
    }
    // a batch of one key has its root at level 0
    for (int i = 0; i < nb; ++i)
        if (B[g.batch[i]] == 1) g.root_row[i] = g.pre[0][i];
    g.nodes = off;
}

template <int P>
snt_status launch_group(snt_ctx *ctx, const Group &g, uint8_t *tables, cudaStream_t st,
                        cudaStream_t aux, cudaEvent_t ev_fork, cudaEvent_t ev_join, int lanes,
                        int split, bool mma, int tiles, int kpt) {
    const ParamInfo &pi = g.pi;
    const int nb = (int)g.batch.size();
    int16_t *nodes = reinterpret_cast<int16_t *>(ctx->arena + g.off_nodes);
    int8_t *gbuf = reinterpret_cast<int8_t *>(ctx->arena + g.off_g);
    int *fix_count = reinterpret_cast<int *>(ctx->arena + g.off_fix);
    int *fix_keys = fix_count + 1;
    int8_t *gfix = reinterpret_cast<int8_t *>(ctx->arena + g.off_gfix);
    KeyMap km;
    std::memset(&km, 0, sizeof(km));
    km.tab = reinterpret_cast<const BatchDesc *>(tables + g.t_desc);
    km.nb = nb;
    const int *pre = reinterpret_cast<const int *>(tables + g.t_pre);  // [level][nb + 1]
    const int *roots = reinterpret_cast<const int *>(tables + g.t_root);
    const int sb = pi.small_bytes;
    // g's first draw with f; the R/3 inversions run beside the whole forest
    // and are joined at the end, before the fix-up of resampled keys
    SNT_CUDA_R(launch_sample_f<P>(km, g.nkeys, nodes, pi.sk_bytes, 2 * sb + pi.pk_bytes, st, gbuf,
                                  nullptr, nullptr, 0, fix_count));
    SNT_CUDA_R(cudaEventRecord(ev_fork, st));
    SNT_CUDA_R(cudaStreamWaitEvent(aux, ev_fork, 0));
    SNT_CUDA_R(launch_r3_keygen<P>(km, g.nkeys, gbuf, pi.sk_bytes, sb, nullptr, nullptr, 0,
                                   ctx->d_err, aux, lanes, kpt, gfix, fix_count, fix_keys));
    SNT_CUDA_R(cudaEventRecord(ev_join, aux));
    for (int l = 1; l <= g.L; ++l) {
        LevelMap lm;
        lm.pre_in = pre + (size_t)(l - 1) * (nb + 1);
        lm.pre_out = pre + (size_t)l * (nb + 1);
        lm.nb = nb;
        lm.n_in = 0;
        const int n_out = g.pre[l][nb];
        if (mma)
            SNT_CUDA_R(launch_tree_up_mma<P>(nodes + (size_t)g.lev_off[l - 1] * pi.pad, lm, n_out,
                                             nodes + (size_t)g.lev_off[l] * pi.pad, st, tiles,
                                             l == 1, ctx->mma_ksplit));
        else
            SNT_CUDA_R(launch_tree_up<P>(nodes + (size_t)g.lev_off[l - 1] * pi.pad, lm, n_out,
                                         nodes + (size_t)g.lev_off[l] * pi.pad, st, split));
    }
    SNT_CUDA_R(launch_rq_inv_jump<P>(nb, nodes, pi.pad, nodes, pi.pad, nullptr, ctx->d_err,
                                     ERR_ROOT, st, roots));
    for (int l = g.L; l >= 1; --l) {
        LevelMap lm;
        lm.pre_in = pre + (size_t)(l - 1) * (nb + 1);
        lm.pre_out = pre + (size_t)l * (nb + 1);
        lm.nb = nb;
        lm.n_in = 0;
        const int n_par = g.pre[l][nb];
        if (mma)
            SNT_CUDA_R(launch_tree_down_mma<P>(nodes + (size_t)g.lev_off[l] * pi.pad, lm, n_par,
                                               nodes + (size_t)g.lev_off[l - 1] * pi.pad, st,
                                               tiles, l == 1, ctx->mma_ksplit));
        else
            SNT_CUDA_R(launch_tree_down<P>(nodes + (size_t)g.lev_off[l] * pi.pad, lm, n_par,
                                           nodes + (size_t)g.lev_off[l - 1] * pi.pad, st, split));
    }
    SNT_CUDA_R(launch_finalize<P>(km, g.nkeys, gbuf, nodes, pi.pk_bytes, pi.sk_bytes, 2 * sb,
                                  pi.sched, st, mma));
    SNT_CUDA_R(launch_sha512_pk(km, g.nkeys, pi.pk_bytes, pi.sk_bytes, 3 * sb + pi.pk_bytes, st));
    SNT_CUDA_R(cudaStreamWaitEvent(st, ev_join, 0));
    SNT_CUDA_R(launch_fixup<P>(km, fix_count, fix_keys, gfix, nodes, pi.pk_bytes, pi.sk_bytes,
                               2 * sb, 3 * sb + pi.pk_bytes, pi.sched, st));
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
        plan_group(g, B);
        g.off_nodes = arena_off;
        arena_off += align_up(g.nodes * g.pi.pad * sizeof(int16_t), 256);
        g.off_g = arena_off;
        arena_off += align_up((size_t)g.nkeys * g.pi.pad, 256);
        g.off_fix = arena_off;
        arena_off += align_up(sizeof(int) * (1 + (size_t)g.nkeys), 256);
        g.off_gfix = arena_off;
        arena_off += align_up((size_t)g.nkeys * g.pi.pad, 256);
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
    // per-call data first (pageable source: staged before the call returns)
    SNT_CUDA_R(cudaMemcpyAsync(tables, host.data(), tbytes, cudaMemcpyHostToDevice, caller));

    std::vector<int> sig;
    sig.reserve(2 * n_batches);
    for (size_t i = 0; i < n_batches; ++i) {
        sig.push_back(P[i]);
        sig.push_back((int)B[i]);
    }
    RaggedGraph &rg = ctx->ragged;
    const int lanes = ctx->r3_lanes, split = ctx->tree_split, tiles = ctx->mma_tiles;
    const int kpt = ctx->r3_kpt;
    const bool mma = ctx->rq_engine != 0;
    // the cached graph holds the kernel layouts: they are part of its key
    sig.push_back(lanes);
    sig.push_back(split);
    sig.push_back(mma ? tiles : 0);
    sig.push_back(kpt);
    sig.push_back(ctx->mma_ksplit);
    if (!(rg.exec && rg.sig == sig && rg.table_off == table_off)) {
        if (rg.exec) cudaGraphExecDestroy(rg.exec);
        rg.exec = nullptr;
        rg.sig.clear();
        // capture the launches of every group on the tree stream (R/3 forks
        // to the auxiliary stream inside the capture)
        SNT_CUDA_R(cudaStreamBeginCapture(ctx->tree, cudaStreamCaptureModeThreadLocal));
        snt_status s = SNT_OK;
        for (int j = 0; j < 3 && s == SNT_OK; ++j) {
            const Group &g = groups[j];
            if (g.batch.empty()) continue;
            switch (g.P) {
                case 653: s = launch_group<653>(ctx, g, tables, ctx->tree, ctx->aux, ctx->ev_fork, ctx->ev_join, lanes, split, mma, tiles, kpt); break;
                case 761: s = launch_group<761>(ctx, g, tables, ctx->tree, ctx->aux, ctx->ev_fork, ctx->ev_join, lanes, split, mma, tiles, kpt); break;
                default: s = launch_group<857>(ctx, g, tables, ctx->tree, ctx->aux, ctx->ev_fork, ctx->ev_join, lanes, split, mma, tiles, kpt); break;
            }
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(ctx->tree, &graph);
        if (s != SNT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
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
