// serve.cu -- the serving loop: a device-resident key pool refilled by batch
// key generation, and continuous batching of encapsulation / decapsulation
// requests (snt_serve_run).
//
// The paper's engNTRU middleware keeps a per-parameter-set pool of key pairs
// filled by the batch call, serves each request from it and refills it when
// it runs empty (Sec. 4.2, batch_lib).  Here the pool lives in device memory
// as chunks of `refill_batch` keys; a chunk whose keys have all been used is
// regenerated by batch keygen on a low-priority stream while requests
// continue.
//
// Workload (a stream of handshakes): encapsulation requests arrive as a
// Poisson process; each item takes a fresh pool key (the one-time key of a
// handshake) and produces a ciphertext.  With probability dec_fraction the
// request is followed by a decapsulation request for the same items, which
// arrives when the encapsulation completes; its session keys are checked
// against the encapsulation's (dec(enc(pk)) = ss).  A key is used up when
// its ciphertext has been decapsulated, or when its encapsulation completes
// if no decapsulation follows.
//
// Continuous batching: requests wait in one FIFO per type; whenever a launch
// slot (stream) is free, the loop admits the oldest requests across both
// FIFOs while launch items, pool keys and the memory budget allow, builds one
// item table for all of them and launches the encapsulation and
// decapsulation kernels on the slot's stream.  Up to `max_inflight` launches
// run concurrently.  Latency is measured per request from its arrival to the
// completion of the launch holding its last item.
//
// Progress: keys are handed out in ring order over the chunks, so at most one
// chunk (the current one) is partly handed out.  An encapsulation request is
// admitted whole; a decapsulation request needs no key and may be split over
// launches.  Every key handed out is used up by work that is always
// admissible (the launch in flight, then the decapsulation that follows), so
// every chunk but the current one is eventually refilled, and since a chunk
// holds at least max_items keys the head encapsulation then fits.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <numeric>
#include <random>
#include <vector>

#include "ctx.h"

using namespace snt;

namespace {

#define SNT_CUDA_V(call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            st = set_error(SNT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));            \
            goto done;                                                                     \
        }                                                                                  \
    } while (0)

struct Request {
    double arrival = -1, finish = -1;
    int type = 0;            // 0 encapsulation, 1 decapsulation
    int n = 0;               // items
    int left = 0;            // items not yet admitted
    int parts = 0;           // launches in flight holding items of this request
    int dec = -1;            // encapsulation: index of the decapsulation that follows, or -1
    std::vector<int> slots;  // pool slots of the items
};

struct Launch {
    bool busy = false;
    std::vector<int> reqs;                  // requests with items in this launch
    std::vector<int> enc_slots, enc_owner;  // per encapsulation item: pool slot, request
    std::vector<int> dec_slots;             // per decapsulation item: pool slot
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    EncItem *d_enc = nullptr;
    DecItem *d_dec = nullptr;
    uint8_t *d_ss = nullptr;  // launch-local session keys (enc items, then dec items)
    EncItem *h_enc = nullptr;
    DecItem *h_dec = nullptr;
    uint8_t *h_ss = nullptr;
};

struct Chunk {
    int state = 0;  // 0 free, 1 filling, 2 ready
    int next = 0;   // keys handed out
    int done = 0;   // keys used up
};

double pct(std::vector<double> v, double q) {
    if (v.empty()) return 0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" snt_status snt_serve_run(snt_ctx *ctx, const snt_serve_config *cfg,
                                    snt_serve_stats *out, double *latency_ms,
                                    size_t latency_cap, snt_serve_audit *audit) {
    if (!ctx || !cfg || !out) return set_error(SNT_EINVAL, "null argument");
    ParamInfo pi;
    if (!param_info(cfg->P, pi)) return set_error(SNT_EINVAL, "unknown parameter set %d", cfg->P);
    if (cfg->rate <= 0 || cfg->duration_s <= 0 || cfg->max_items < 1 || cfg->max_inflight < 1 ||
        cfg->refill_batch < (size_t)cfg->max_items || cfg->refill_batch > 8192 ||
        cfg->max_launch_items < cfg->max_items || cfg->max_launch_items < 64)
        return set_error(SNT_EINVAL, "bad serving configuration");
    const int chunk = (int)cfg->refill_batch;
    const int nchunk = (int)std::max<size_t>(2, cfg->pool_keys / cfg->refill_batch);
    const int cap = nchunk * chunk;
    const int L = cfg->max_launch_items;
    const int S = cfg->max_inflight;
    const size_t pkb = pi.pk_bytes, skb = pi.sk_bytes, ctb = pi.ct_bytes;
    if (audit) {
        if (audit->cap && (!audit->k || !audit->pk || !audit->ct || !audit->ss))
            return set_error(SNT_EINVAL, "audit buffers missing");
        audit->count = 0;
    }
    // device memory: pool (pk, sk, ct per key) and per-launch item tables
    const size_t pool_bytes = align256((size_t)cap * (pkb + skb + ctb));
    const size_t launch_bytes = align256((size_t)L * (sizeof(EncItem) + sizeof(DecItem) + 32));
    const size_t need = pool_bytes + (size_t)S * launch_bytes;
    if (need > cfg->mem_budget)
        return set_error(SNT_ENOMEM, "serving state needs %zu bytes, budget %zu", need, cfg->mem_budget);
    if (keygen_arena(pi, (size_t)chunk, false) > ctx->budget)
        return set_error(SNT_ENOMEM, "refill batch of %d keys exceeds the context budget", chunk);

    DeviceGuard dg(ctx->device);
    snt_status st = SNT_OK;
    uint8_t *dmem = nullptr;
    std::vector<Launch> ls(S);
    cudaStream_t refill = nullptr;
    cudaEvent_t ev_refill = nullptr;
    std::vector<Request> reqs;
    std::vector<int> enc_order;  // encapsulation requests in arrival order
    std::vector<uint8_t> ss_enc((size_t)cap * 32);
    std::vector<Chunk> chunks(nchunk);
    std::deque<int> qenc, qdec;
    int refilling = -1;
    int cur = 0;  // chunk keys are handed out from (ring order)
    uint64_t key_counter = 0, enc_counter = 0;
    size_t mism = 0, items_enc = 0, items_dec = 0, keys_generated = 0, mem_waits = 0;
    size_t inflight_items = 0, max_queue = 0, finished = 0;
    size_t budget_items = 0;
    double t_end = 0;
    int prio_low = 0, prio_high = 0;
    uint8_t *pool_pk = nullptr, *pool_sk = nullptr, *pool_ct = nullptr;
    std::mt19937_64 rng(cfg->seed);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    using clk = std::chrono::steady_clock;
    clk::time_point t0;
    // a key is used up: its chunk is free for a refill once all its keys are
    auto key_done = [&](int slot) {
        Chunk &ch = chunks[slot / chunk];
        if (++ch.done == chunk) { ch.state = 0; ch.next = 0; ch.done = 0; }
    };
    // next pool key; the caller has checked that a ready key exists.  Only
    // the current chunk can be partly handed out, so every other ready chunk
    // is untouched and the first one after `cur` in ring order takes over.
    auto take_key = [&]() -> int {
        if (!(chunks[cur].state == 2 && chunks[cur].next < chunk)) {
            int c = cur;
            for (int i = 0; i < nchunk; ++i) {
                c = (c + 1) % nchunk;
                if (chunks[c].state == 2 && chunks[c].next == 0) break;
            }
            cur = c;
        }
        return cur * chunk + chunks[cur].next++;
    };

    SNT_CUDA_V(cudaMalloc(&dmem, need));
    pool_pk = dmem;
    pool_sk = pool_pk + (size_t)cap * pkb;
    pool_ct = pool_sk + (size_t)cap * skb;
    SNT_CUDA_V(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    SNT_CUDA_V(cudaStreamCreateWithPriority(&refill, cudaStreamNonBlocking, prio_low));
    SNT_CUDA_V(cudaEventCreateWithFlags(&ev_refill, cudaEventDisableTiming));
    for (int s = 0; s < S; ++s) {
        Launch &l = ls[s];
        uint8_t *base = dmem + pool_bytes + (size_t)s * launch_bytes;  // 256-aligned
        l.d_enc = reinterpret_cast<EncItem *>(base);
        l.d_dec = reinterpret_cast<DecItem *>(base + (size_t)L * sizeof(EncItem));
        l.d_ss = base + (size_t)L * (sizeof(EncItem) + sizeof(DecItem));
        SNT_CUDA_V(cudaStreamCreateWithPriority(&l.stream, cudaStreamNonBlocking, prio_high));
        SNT_CUDA_V(cudaEventCreateWithFlags(&l.ev, cudaEventDisableTiming));
        SNT_CUDA_V(cudaMallocHost(&l.h_enc, (size_t)L * sizeof(EncItem)));
        SNT_CUDA_V(cudaMallocHost(&l.h_dec, (size_t)L * sizeof(DecItem)));
        SNT_CUDA_V(cudaMallocHost(&l.h_ss, (size_t)L * 32));
    }
    // the item memory the budget leaves for in-flight work: each in-flight
    // item holds one ciphertext-sized slot of the launch tables and results
    budget_items = (cfg->mem_budget - pool_bytes) / (ctb + 32 + sizeof(EncItem));

    {   // encapsulation arrivals: Poisson at rate / (1 + dec_fraction), so that
        // the request stream (with the decapsulations) averages `rate`; sizes
        // log-uniform in [1, max_items]
        const double f = std::min(1.0, std::max(0.0, cfg->dec_fraction));
        const double rate_enc = cfg->rate / (1.0 + f);
        double t = 0;
        for (;;) {
            t += -std::log(1.0 - U(rng)) / rate_enc;
            if (t >= cfg->duration_s) break;
            Request r;
            r.arrival = t;
            r.type = 0;
            r.n = std::min(cfg->max_items, (int)std::floor(std::exp(U(rng) * std::log(cfg->max_items + 1.0))));
            r.n = std::max(1, r.n);
            r.left = r.n;
            const bool with_dec = U(rng) < f;
            enc_order.push_back((int)reqs.size());
            reqs.push_back(r);
            if (with_dec) {
                reqs.back().dec = (int)reqs.size();
                Request d;
                d.type = 1;
                d.n = r.n;
                reqs.push_back(d);
            }
        }
    }

    // the pool starts full (the batch call on first use)
    for (int c = 0; c < nchunk; ++c) {
        const snt_status s2 = keygen_into(ctx, cfg->P, cfg->seed, key_counter, (size_t)chunk,
                                          pool_pk + (size_t)c * chunk * pkb,
                                          pool_sk + (size_t)c * chunk * skb, refill);
        if (s2 != SNT_OK) { st = s2; goto done; }
        key_counter += chunk;
        chunks[c].state = 2;
    }
    SNT_CUDA_V(cudaStreamSynchronize(refill));

    t0 = clk::now();
    {
        size_t next_arr = 0;
        auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
        const double give_up = cfg->duration_s + 20.0;
        while (finished < reqs.size()) {
            const double t = now_s();
            if (t > give_up) {
                int avail = 0, busy = 0;
                char cs[64] = {0};
                for (int c = 0; c < nchunk && c < 60; ++c) {
                    if (chunks[c].state == 2) avail += chunk - chunks[c].next;
                    cs[c] = (char)('0' + chunks[c].state);
                }
                for (int s = 0; s < S; ++s) busy += ls[s].busy;
                st = set_error(SNT_ETIMEOUT,
                               "serving run did not drain within %.0f s: %zu/%zu finished, queues "
                               "enc %zu dec %zu, free keys %d, chunks %s, refilling %d, busy launches %d",
                               give_up, finished, reqs.size(), qenc.size(), qdec.size(), avail, cs,
                               refilling, busy);
                goto done;
            }
            while (next_arr < enc_order.size() && reqs[enc_order[next_arr]].arrival <= t)
                qenc.push_back(enc_order[next_arr++]);
            max_queue = std::max(max_queue, qenc.size() + qdec.size());
            // completions
            for (int s = 0; s < S; ++s) {
                Launch &l = ls[s];
                if (!l.busy) continue;
                const cudaError_t q = cudaEventQuery(l.ev);
                if (q == cudaErrorNotReady) continue;
                SNT_CUDA_V(q);
                const double tf = now_s();
                const int ne = (int)l.enc_slots.size();
                for (int i = 0; i < ne; ++i) {
                    const int slot = l.enc_slots[i];
                    std::memcpy(&ss_enc[(size_t)slot * 32], l.h_ss + 32 * i, 32);
                    if (reqs[l.enc_owner[i]].dec < 0) key_done(slot);
                    if (audit && audit->count < audit->cap) {  // record for the caller
                        const size_t a = audit->count++;
                        audit->k[a] = l.h_enc[i].k;
                        std::memcpy(audit->ss + a * 32, l.h_ss + 32 * i, 32);
                        SNT_CUDA_V(cudaMemcpy(audit->pk + a * pkb, pool_pk + (size_t)slot * pkb, pkb, cudaMemcpyDeviceToHost));
                        SNT_CUDA_V(cudaMemcpy(audit->ct + a * ctb, pool_ct + (size_t)slot * ctb, ctb, cudaMemcpyDeviceToHost));
                    }
                }
                for (size_t i = 0; i < l.dec_slots.size(); ++i) {
                    const int slot = l.dec_slots[i];
                    if (std::memcmp(&ss_enc[(size_t)slot * 32], l.h_ss + 32 * (ne + i), 32) != 0) ++mism;
                    key_done(slot);
                }
                for (int r : l.reqs) {
                    Request &rq = reqs[r];
                    if (--rq.parts > 0 || rq.left > 0) continue;
                    rq.finish = tf;
                    ++finished;
                    if (rq.type == 0 && rq.dec >= 0) {  // the handshake's decapsulation arrives
                        Request &d = reqs[rq.dec];
                        d.arrival = tf;
                        d.slots = rq.slots;
                        d.left = d.n;
                        qdec.push_back(rq.dec);
                    }
                }
                inflight_items -= l.enc_slots.size() + l.dec_slots.size();
                l.busy = false;
                l.reqs.clear();
                l.enc_slots.clear();
                l.enc_owner.clear();
                l.dec_slots.clear();
            }
            // refill
            if (refilling >= 0) {
                const cudaError_t q = cudaEventQuery(ev_refill);
                if (q != cudaErrorNotReady) {
                    SNT_CUDA_V(q);
                    chunks[refilling].state = 2;
                    refilling = -1;
                }
            }
            if (refilling < 0) {
                for (int c = 0; c < nchunk; ++c)
                    if (chunks[c].state == 0) {
                        const snt_status s2 = keygen_into(ctx, cfg->P, cfg->seed, key_counter, (size_t)chunk,
                                                          pool_pk + (size_t)c * chunk * pkb,
                                                          pool_sk + (size_t)c * chunk * skb, refill);
                        if (s2 != SNT_OK) { st = s2; goto done; }
                        SNT_CUDA_V(cudaEventRecord(ev_refill, refill));
                        key_counter += chunk;
                        keys_generated += chunk;
                        chunks[c].state = 1;
                        refilling = c;
                        break;
                    }
            }
            // admission and launch
            int free_slot = -1;
            for (int s = 0; s < S; ++s)
                if (!ls[s].busy) { free_slot = s; break; }
            if (free_slot >= 0 && (!qenc.empty() || !qdec.empty())) {
                Launch &l = ls[free_slot];
                int ne = 0, nd = 0;
                int avail = 0;
                for (int c = 0; c < nchunk; ++c)
                    if (chunks[c].state == 2) avail += chunk - chunks[c].next;
                size_t budget_left = budget_items > inflight_items ? budget_items - inflight_items : 0;
                // oldest request first across the two FIFOs; an encapsulation
                // needs pool keys, a decapsulation only its own ciphertexts
                while (ne + nd < L) {
                    const bool eok = !qenc.empty() && avail >= reqs[qenc.front()].left;
                    const bool dok = !qdec.empty();
                    if (!eok && !dok) break;
                    const bool take_dec =
                        dok && (!eok || reqs[qdec.front()].arrival <= reqs[qenc.front()].arrival);
                    const int qi = take_dec ? qdec.front() : qenc.front();
                    Request &r = reqs[qi];
                    int k = std::min(r.left, L - ne - nd);
                    if (!take_dec && k < r.left) break;  // encapsulations are admitted whole
                    bool limited = false;
                    if ((size_t)k > budget_left) {
                        ++mem_waits;
                        if (!take_dec) break;
                        k = (int)budget_left;
                        limited = true;
                    }
                    if (k <= 0) break;
                    if (take_dec) {
                        const int off = r.n - r.left;
                        for (int i = 0; i < k; ++i) l.dec_slots.push_back(r.slots[off + i]);
                        nd += k;
                    } else {
                        for (int i = 0; i < k; ++i) {
                            const int slot = take_key();
                            r.slots.push_back(slot);
                            l.enc_slots.push_back(slot);
                            l.enc_owner.push_back(qi);
                        }
                        avail -= k;
                        ne += k;
                    }
                    budget_left -= (size_t)k;
                    r.left -= k;
                    ++r.parts;
                    l.reqs.push_back(qi);
                    if (r.left == 0) (take_dec ? qdec : qenc).pop_front();
                    if (limited) break;
                }
                if (!l.reqs.empty()) {
                    for (int i = 0; i < ne; ++i) {
                        const int slot = l.enc_slots[i];
                        l.h_enc[i].pk = pool_pk + (size_t)slot * pkb;
                        l.h_enc[i].cache = pool_sk + (size_t)slot * skb + (skb - 32);
                        l.h_enc[i].k = enc_counter++;
                        l.h_enc[i].ct = pool_ct + (size_t)slot * ctb;
                        l.h_enc[i].ss = l.d_ss + (size_t)i * 32;
                    }
                    for (int i = 0; i < nd; ++i) {
                        const int slot = l.dec_slots[i];
                        l.h_dec[i].sk = pool_sk + (size_t)slot * skb;
                        l.h_dec[i].ct = pool_ct + (size_t)slot * ctb;
                        l.h_dec[i].ss = l.d_ss + (size_t)(ne + i) * 32;
                    }
                    if (ne) SNT_CUDA_V(cudaMemcpyAsync(l.d_enc, l.h_enc, (size_t)ne * sizeof(EncItem), cudaMemcpyHostToDevice, l.stream));
                    if (nd) SNT_CUDA_V(cudaMemcpyAsync(l.d_dec, l.h_dec, (size_t)nd * sizeof(DecItem), cudaMemcpyHostToDevice, l.stream));
                    EncMap em;
                    std::memset(&em, 0, sizeof(em));
                    em.tab = l.d_enc;
                    em.seed = cfg->seed;
                    DecMap dm;
                    std::memset(&dm, 0, sizeof(dm));
                    dm.tab = l.d_dec;
                    cudaError_t e = cudaSuccess;
                    switch (cfg->P) {
                        case 653:
                            if (ne) e = launch_encap<653>(em, ne, (int)pkb, (int)ctb, pi.sched, pi.rsched, l.stream);
                            if (nd && e == cudaSuccess) e = launch_decap<653>(dm, nd, (int)pkb, (int)skb, (int)ctb, pi.sched, pi.rsched, l.stream);
                            break;
                        case 761:
                            if (ne) e = launch_encap<761>(em, ne, (int)pkb, (int)ctb, pi.sched, pi.rsched, l.stream);
                            if (nd && e == cudaSuccess) e = launch_decap<761>(dm, nd, (int)pkb, (int)skb, (int)ctb, pi.sched, pi.rsched, l.stream);
                            break;
                        default:
                            if (ne) e = launch_encap<857>(em, ne, (int)pkb, (int)ctb, pi.sched, pi.rsched, l.stream);
                            if (nd && e == cudaSuccess) e = launch_decap<857>(dm, nd, (int)pkb, (int)skb, (int)ctb, pi.sched, pi.rsched, l.stream);
                            break;
                    }
                    SNT_CUDA_V(e);
                    SNT_CUDA_V(cudaMemcpyAsync(l.h_ss, l.d_ss, (size_t)(ne + nd) * 32, cudaMemcpyDeviceToHost, l.stream));
                    SNT_CUDA_V(cudaEventRecord(l.ev, l.stream));
                    l.busy = true;
                    inflight_items += ne + nd;
                    items_enc += ne;
                    items_dec += nd;
                }
            }
        }
        t_end = now_s();
    }

    {
        std::vector<double> lat;
        lat.reserve(reqs.size());
        for (size_t i = 0; i < reqs.size(); ++i) {
            const double ms = 1e3 * (reqs[i].finish - reqs[i].arrival);
            lat.push_back(ms);
            if (latency_ms && i < latency_cap) latency_ms[i] = ms;
        }
        std::memset(out, 0, sizeof(*out));
        out->requests = reqs.size();
        out->items_enc = items_enc;
        out->items_dec = items_dec;
        out->keys_generated = keys_generated;
        out->mismatches = mism;
        out->memory_waits = mem_waits;
        out->max_queue = max_queue;
        out->wall_s = t_end;
        out->p50_ms = pct(lat, 0.50);
        out->p99_ms = pct(lat, 0.99);
        out->mean_ms = lat.empty() ? 0 : std::accumulate(lat.begin(), lat.end(), 0.0) / (double)lat.size();
        out->max_ms = lat.empty() ? 0 : *std::max_element(lat.begin(), lat.end());
        out->items_per_s = t_end > 0 ? (double)(items_enc + items_dec) / t_end : 0;
        out->requests_per_s = t_end > 0 ? (double)reqs.size() / t_end : 0;
    }
    st = snt_ctx_sync(ctx, refill);

done:
    for (Launch &l : ls) {
        if (l.stream) cudaStreamSynchronize(l.stream);
        if (l.ev) cudaEventDestroy(l.ev);
        if (l.stream) cudaStreamDestroy(l.stream);
        if (l.h_enc) cudaFreeHost(l.h_enc);
        if (l.h_dec) cudaFreeHost(l.h_dec);
        if (l.h_ss) cudaFreeHost(l.h_ss);
    }
    if (refill) { cudaStreamSynchronize(refill); cudaStreamDestroy(refill); }
    if (ev_refill) cudaEventDestroy(ev_refill);
    if (dmem) { cudaMemset(dmem, 0, need); cudaDeviceSynchronize(); cudaFree(dmem); }
    return st;
}
