/*
 * sntrup_gb300.h -- C ABI of the GB300 (sm_103a) batch key generation library
 * for Streamlined NTRU Prime (sntrup653, sntrup761, sntrup857).
 *
 * Method: arXiv 2106.08759 ("OpenSSLNTRU: Faster post-quantum TLS key
 * exchange"), Sec. 3.1 KeyGen and Algorithm 1 (BatchKeyGen): per key a small g
 * invertible in R/3 and a Short f; v = 1/g in R/3; the inverses of all 3f in
 * R/q at once by Montgomery's trick (Sec. 2.2), run as a product tree with one
 * root inversion; h = g / (3f); pk = Rq_encode(h); sk = Small_encode(f) |
 * Small_encode(v) | pk | rho | Hash_prefix(4, pk).
 *
 * Conventions shared by every call:
 *   - All functions return snt_status: SNT_OK (0) or a negative code.  On any
 *     error the output buffers are undefined and must not be used;
 *     snt_last_error_string() gives a one-line reason (per host thread).
 *   - Buffers named *_dev are device pointers on the context's device, owned
 *     by the caller; *_host are host pointers owned by the caller.  The library
 *     owns only the scratch memory inside a context.
 *   - Calls taking a stream are asynchronous on that stream (NULL = the legacy
 *     default stream).  Device-side failures (exhausted resampling, a bounded
 *     wait that gave up) are recorded in a per-context error word that
 *     snt_ctx_sync() reads; it returns the failure as SNT_EINTERNAL /
 *     SNT_ETIMEOUT and clears the word.
 *   - A context is used by one host thread at a time.
 *   - Key i of a call uses randomness (seed, first_key_index + i) only, so a
 *     batch split into sub-batches of any sizes yields identical bytes.
 *
 * Randomness (the paper only says "uniform random", Algorithm 1): word j of
 * stream s at attempt a for key index k is lane (j mod 4) of Philox4x32-10
 * with key (seed mod 2^32, seed >> 32) and counter ((s << 16) | (j / 4), a,
 * k mod 2^32, k >> 32); stream 0 draws g, 1 draws f, 2 draws rho.
 */
#ifndef SNTRUP_GB300_H
#define SNTRUP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SNT_OK = 0,
    SNT_EINVAL = -1,     /* null pointer, zero or oversized count, unknown parameter set */
    SNT_ENOMEM = -2,     /* request exceeds the context's memory budget */
    SNT_ECUDA = -3,      /* a CUDA runtime call failed */
    SNT_ETIMEOUT = -4,   /* a bounded device-side wait gave up */
    SNT_EINTERNAL = -5   /* device self-check failed (e.g. g resampling exhausted) */
} snt_status;

/* Parameter sets (p, q, w), Sec. 2.1: (653,4621,288), (761,4591,286), (857,5167,322). */
typedef enum { SNTRUP653 = 653, SNTRUP761 = 761, SNTRUP857 = 857 } snt_param;

typedef struct snt_ctx snt_ctx;
typedef struct CUstream_st *snt_stream; /* same type as cudaStream_t */

/* Byte sizes of one public key, secret key, ciphertext and session key.
 * For sntrup761: 1158, 1763, 1039, 32.  pk + sk matches the per-key storage of
 * Table 4 (2512 / 2921 / 3321 bytes); any pointer may be NULL. */
snt_status snt_param_sizes(int P, size_t *pk_bytes, size_t *sk_bytes,
                           size_t *ct_bytes, size_t *ss_bytes);

/* Create a context on CUDA device `device` whose scratch memory never exceeds
 * mem_budget bytes (0 selects 256 MiB).  Scratch is allocated once, here.
 * The largest batch a context accepts is reported by snt_ctx_max_batch. */
snt_status snt_ctx_create(int device, size_t mem_budget, snt_ctx **out);

/* Zero the context's secret-bearing scratch, wait for its work, free it. */
snt_status snt_ctx_destroy(snt_ctx *ctx);

/* Largest B accepted by the keygen calls of this context for parameter set P. */
snt_status snt_ctx_max_batch(snt_ctx *ctx, int P, size_t *max_B);

/* Wait for all work the context issued on `stream` (and on its own streams,
 * the host copies of snt_batch_keygen_host_async included) and read (then
 * clear) the device error word.  Returns SNT_OK if no device-side failure
 * occurred. */
snt_status snt_ctx_sync(snt_ctx *ctx, snt_stream stream);

/* Batch key generation (Algorithm 1 with a product tree for batchInv in R/q).
 * Writes B public keys (pk_dev, B * pk_bytes, key-major, contiguous) and B
 * secret keys (sk_dev, B * sk_bytes).  Key i uses key index
 * first_key_index + i.  1 <= B <= snt_ctx_max_batch(P).  Outputs are
 * byte-identical to snt_keygen_perkey and to any split of the batch.  The
 * work forks from `stream` onto the context's own streams (the product tree,
 * the R/3 inversions, the leaf-pair products of h) and joins back into
 * `stream`, so work ordered after the call on `stream` sees every key. */
snt_status snt_batch_keygen(snt_ctx *ctx, int P, uint64_t seed,
                            uint64_t first_key_index, size_t B,
                            uint8_t *pk_dev, uint8_t *sk_dev, snt_stream stream);

/* Same outputs as snt_batch_keygen, computed without batching the R/q
 * inversion: every key inverts its own 3f by divsteps (Sec. 3.1 KeyGen), by
 * default jump divsteps in one CTA per key (SNT_OPT_PERKEY_INV), and its own
 * 1/g in R/3 by bit-sliced divsteps.  The GPU baseline of the batched path. */
snt_status snt_keygen_perkey(snt_ctx *ctx, int P, uint64_t seed,
                             uint64_t first_key_index, size_t B,
                             uint8_t *pk_dev, uint8_t *sk_dev, snt_stream stream);

/* Many batches in one launch (the ragged workload: uneven sizes, mixed
 * parameter sets).  Batch i has parameter set P[i], B[i] keys with key indices
 * first_idx[i] + j and seed seeds[i], written to pk_dev[i] / sk_dev[i] (device
 * pointers, each B[i] * sizes of P[i]).  Every batch gets exactly the bytes
 * snt_batch_keygen would give it alone: each batch keeps its own Montgomery
 * product tree (Algorithm 1), while the batches of one parameter set share the
 * launches, level by level, and the three parameter sets run side by side on
 * streams of the context.  The R/3 inverses are per key (SNT_OPT_R3_MODE 0)
 * or batched after the invertibility test of Sec. 3.1.1 (modes 1 and 2).  A
 * parameter set takes the layouts snt_autotune_ex chose on this context for
 * (P, the ceil(log2) bucket of its largest batch), else the context's
 * options.  The launch sequence of a plan (the list of (P[i], B[i]) and the
 * layouts) is captured into a CUDA graph on first use and replayed while the
 * plan repeats.  Asynchronous on `stream`; 1 <= n_batches <= 65536. */
snt_status snt_batch_keygen_ragged(snt_ctx *ctx, size_t n_batches, const int *P,
                                   const size_t *B, const uint64_t *seeds,
                                   const uint64_t *first_idx, uint8_t *const *pk_dev,
                                   uint8_t *const *sk_dev, snt_stream stream);

/* Host-memory convenience form of snt_batch_keygen: generates on the device,
 * copies B * pk_bytes and B * sk_bytes into the caller's host buffers and
 * returns when they are complete (synchronous; includes snt_ctx_sync). */
snt_status snt_batch_keygen_host(snt_ctx *ctx, int P, uint64_t seed,
                                 uint64_t first_key_index, size_t B,
                                 uint8_t *pk_host, uint8_t *sk_host);

/* The same into host memory without waiting: enqueues the generation on
 * `stream` (as snt_batch_keygen, into a staging slot of the context's
 * scratch) and the two device-to-host copies on the context's copy streams,
 * and returns.  The keys are in pk_host / sk_host once snt_ctx_sync(ctx,
 * stream) has returned SNT_OK.  With room in the budget for two staging
 * slots (snt_ctx_max_batch counts one) consecutive calls alternate between
 * them, so one call's copies overlap the next call's generation; a call
 * waits on the device for the copies of the call that last used its slot.
 * pk_host / sk_host should be page-locked (cudaHostAlloc or registered) for
 * the copies to run asynchronously; they must stay valid and untouched
 * until the sync.  Errors of the arguments are returned at once, device
 * errors by the sync. */
snt_status snt_batch_keygen_host_async(snt_ctx *ctx, int P, uint64_t seed,
                                       uint64_t first_key_index, size_t B, uint8_t *pk_host,
                                       uint8_t *sk_host, snt_stream stream);

/* Batch key generation for callers that cannot allocate device memory (the
 * paper has no counterpart; it is a deployment variant of snt_batch_keygen).
 * Who needs it: code running while a framework's caching allocator owns the
 * free device memory, latency-bound paths where cudaMalloc / cudaFree would
 * synchronise the device, and processes that may not allocate after start-up.
 * It takes no context and allocates nothing: its scratch is a fixed 1152 KiB
 * static device array inside this library, which every GPU that loads the
 * library holds until the process exits.
 *   - 1 <= B <= 256 keys per call; larger B returns SNT_EINVAL with a message.
 *   - Writes the same bytes as snt_batch_keygen (same pk/sk layout).
 *   - The first call on a device looks up the scratch array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make
 *     that first call before any stream capture on the device.  The cached
 *     address lives as long as the device's primary context: do not call
 *     cudaDeviceReset on a device while this library stays loaded.
 *   - Every call uses the same scratch, which keeps the previous call's data:
 *     calls whose GPU work overlaps (different streams, threads or processes
 *     sharing the library instance without ordering) race and corrupt each
 *     other's keys.  Order them on one stream or synchronise in between.
 *   - Returns after the keys are written: it waits for `stream` in order to
 *     report device-side failures (SNT_EINTERNAL).  No host thread may call it
 *     concurrently for the same device. */
snt_status snt_batch_keygen_static(int device, int P, uint64_t seed,
                                   uint64_t first_key_index, size_t B,
                                   uint8_t *pk_dev, uint8_t *sk_dev, snt_stream stream);

/* ---- Key encapsulation (the serving path) ----
 * The paper measures encapsulation and decapsulation (Table 1: 46914 and 56241
 * Haswell cycles for sntrup761) and takes their definition from the NTRU
 * Prime specification.  Reading (round-3 Streamlined NTRU Prime KEM): the
 * ciphertext is Rounded_encode(Round(h r)) | Hash_prefix(2, Hash_prefix(3,
 * r_enc) | Hash_prefix(4, pk)) (1039 bytes for sntrup761, Table 1's 2197
 * key + ciphertext bytes), the session key Hash_prefix(1, Hash_prefix(3, r_enc)
 * | ct); decapsulation re-encrypts and falls back to Hash_prefix(0,
 * Hash_prefix(3, rho) | ct) if the ciphertext does not match (implicit
 * rejection).  A CTA runs the ring arithmetic of up to 32 items in turn and
 * one of its warps hashes them, a lane per item (one item per CTA for small
 * counts).  Asynchronous on `stream`. */

/* n encapsulations: item i uses pk_dev + i * pk_bytes and the Short r of
 * stream 3 for (seed, first_idx + i); writes ct_dev + i * ct_bytes and
 * ss_dev + i * 32. */
snt_status snt_enc(snt_ctx *ctx, int P, size_t n, const uint8_t *pk_dev, uint64_t seed,
                   uint64_t first_idx, uint8_t *ct_dev, uint8_t *ss_dev, snt_stream stream);

/* n decapsulations: item i uses sk_dev + i * sk_bytes and ct_dev + i * ct_bytes,
 * writes ss_dev + i * 32. */
snt_status snt_dec(snt_ctx *ctx, int P, size_t n, const uint8_t *sk_dev, const uint8_t *ct_dev,
                   uint8_t *ss_dev, snt_stream stream);

/* ---- Serving loop ----
 * A device-resident pool of key pairs refilled by batch key generation (the
 * pool of the paper's engNTRU batch_lib, Sec. 4.2), and a stream of
 * handshakes served by continuous batching.  Encapsulation requests arrive as
 * a Poisson process; every item takes a fresh pool key.  With probability
 * dec_fraction a request is followed by a decapsulation request for the same
 * items, arriving when the encapsulation completes; its session keys are
 * checked against the encapsulation's.  Arrived requests wait in one FIFO per
 * type and are admitted oldest first as launch slots, pool keys and the
 * memory budget allow (an encapsulation whole, a decapsulation possibly over
 * several launches); up to max_inflight launches run concurrently. */
typedef struct {
    int P;                   /* parameter set */
    double rate;             /* requests per second, both types (encapsulations are
                                Poisson at rate / (1 + dec_fraction)) */
    double duration_s;       /* length of the arrival stream in seconds */
    int max_items;           /* items per request: log-uniform in [1, max_items] */
    double dec_fraction;     /* probability that an encapsulation request is followed
                                by a decapsulation of its items, in [0, 1] */
    size_t pool_keys;        /* key pool capacity (rounded to refill batches, >= 2 of them) */
    size_t refill_batch;     /* keys per refill, in [max_items, 8192] */
    size_t mem_budget;       /* device bytes for the pool and in-flight items */
    int max_inflight;        /* concurrent launches */
    int max_launch_items;    /* items per launch (>= max(64, max_items)) */
    uint64_t seed;           /* keys, encapsulation randomness, arrival process */
} snt_serve_config;

typedef struct {
    size_t requests, items_enc, items_dec, keys_generated;
    size_t mismatches;       /* decapsulations whose key differed from the encapsulation's */
    size_t memory_waits;     /* admissions deferred by the memory budget */
    size_t max_queue;        /* longest request queue seen */
    double wall_s, p50_ms, p99_ms, mean_ms, max_ms, items_per_s, requests_per_s;
} snt_serve_stats;

/* Optional record of the first `cap` encapsulation items served: key index
 * k[i] of the encapsulation randomness (stream 3 of cfg->seed), the public
 * key pk[i * pk_bytes ..], ciphertext ct[i * ct_bytes ..] and session key
 * ss[i * 32 ..] (host buffers of the caller); count is set on return.  Lets a
 * caller recompute those items alone and compare. */
typedef struct {
    size_t cap, count;
    uint64_t *k;
    uint8_t *pk, *ct, *ss;
} snt_serve_audit;

/* Runs the arrival stream in real time and returns latency statistics
 * (arrival to completion of the launch holding the request's last item).  Synchronous.  If
 * latency_ms is not NULL, the latency of request i (arrival order) is written
 * to latency_ms[i] for i < latency_cap; audit may be NULL.  Uses the
 * context's scratch for the refills and allocates the pool (within
 * mem_budget) for the run.  Request order: encapsulation requests by arrival,
 * each followed by its decapsulation request if it has one.  Returns
 * SNT_ETIMEOUT if the requests have not all completed 20 s after the end of
 * the arrival stream. */
snt_status snt_serve_run(snt_ctx *ctx, const snt_serve_config *cfg, snt_serve_stats *out,
                         double *latency_ms, size_t latency_cap, snt_serve_audit *audit);

/* ---- Building blocks (kernel microbenchmarks; same kernels as keygen) ---- */

/* c_i = a_i * b_i in R/q for i < n.  a_dev, b_dev, c_dev: n * p int16
 * coefficients each, key-major, centred in [-(q-1)/2, (q-1)/2] (inputs may
 * be any int16 with |x| <= (q-1)/2); outputs centred. */
snt_status snt_rq_mul(snt_ctx *ctx, int P, size_t n, const int16_t *a_dev,
                      const int16_t *b_dev, int16_t *c_dev, snt_stream stream);

/* out_i = 1/a_i in R/q by divsteps (Bernstein-Yang), one CTA per element.
 * a_dev, out_dev: n * p int16 centred; ok_dev: n int32, 1 if invertible
 * (a_i != 0), else 0 and out_i = 0. */
snt_status snt_rq_inv(snt_ctx *ctx, int P, size_t n, const int16_t *a_dev,
                      int16_t *out_dev, int32_t *ok_dev, snt_stream stream);

/* Same result as snt_rq_inv, latency-optimised (the form used for the single
 * root inversion of the batch tree): jump divsteps, i.e. chunks of 31 steps
 * run by one warp on the low coefficients, whose 2x2 transition matrix the
 * whole CTA then applies (Bernstein-Yang's recursive divsteps, the paper's
 * "jump-div-step" of Table 4's note).  One CTA of 512 threads per element. */
snt_status snt_rq_inv_latency(snt_ctx *ctx, int P, size_t n, const int16_t *a_dev,
                              int16_t *out_dev, int32_t *ok_dev, snt_stream stream);

/* out_i = 1/g_i in R/3 by bit-sliced divsteps, one warp per element.
 * g_dev, out_dev: n * p int8 in {-1,0,1}; ok_dev: n int32, 1 if g_i is
 * invertible in R/3, else 0 and out_i = 0. */
snt_status snt_r3_inv(snt_ctx *ctx, int P, size_t n, const int8_t *g_dev,
                      int8_t *out_dev, int32_t *ok_dev, snt_stream stream);

/* Test hook for the resampling path (Algorithm 1 skips g that fail the
 * invertibility check): for the next keygen calls on this context, attempt 0
 * of key index key_index_host[j] uses g_host[j * p .. j * p + p) (int8 in
 * {-1,0,1}) instead of its random draw.  n = 0 clears the list.  n <= 64. */
snt_status snt_debug_inject_g(snt_ctx *ctx, int P, size_t n,
                              const uint64_t *key_index_host,
                              const int8_t *g_host);

/* ---- Tuning options (kernel layouts; outputs never depend on them) ---- */

typedef enum {
    /* lanes per element of the bit-sliced R/3 divstep kernel: 4, 8 or 32
     * (32 / value elements share a warp) */
    SNT_OPT_R3_LANES = 1,
    /* largest number of thread groups one R/q product of a narrow tree level
     * is split over: 1, 2, 4 or 8 */
    SNT_OPT_TREE_SPLIT = 2,
    /* where the R/3 inversions (per key or batched) run: 0 first, on the
     * tree's stream; 1 on a second stream concurrent with the whole tree; 2
     * on that stream from the up-sweep's first narrow level (fewer than 256
     * products), so they fill the SMs the narrow levels and the root
     * inversion leave idle; 3 on that stream from the end of the up-sweep,
     * so that the R/3 work starts beside the root inversions */
    SNT_OPT_R3_OVERLAP = 3,
    /* 1: each product of a tree level with at most 64 products is split by
     * output segments over several CTAs (up to 12 SMs per product) instead of
     * running on one SM; 0: one CTA per product on every level */
    SNT_OPT_NARROW_SEG = 4,
    /* engine of the R/q products (tree, h excluded, snt_rq_mul): 0 CUDA-core
     * Toeplitz products on the IMAD pipe; 1 the same Toeplitz products on
     * the tensor cores (warp MMA on exact 6-bit f16 limbs, f32 accumulate);
     * 2 the paper's multiplier (Sec. 3.3) on the CUDA cores: truncated
     * transforms over K = (Z/q)[x]/(x^64 + 1) whose twiddles are powers of x
     * (shifts and negations), 48 pointwise products in K for p <= 768 (64 for
     * sntrup857) on the IMAD pipe, for the tree's general x general levels
     * (its leaf levels and h stay on the tensor cores) and snt_rq_mul; 3 the
     * tensor cores with one limb on the vector side of the general products:
     * each residue taken as its representative exact in f16 (an odd residue
     * above 2048 in magnitude moved by q), two MMAs per step instead of four,
     * the f32 partial sums moved into int32 sums every 8 steps */
    SNT_OPT_RQ_ENGINE = 5,
    /* tensor-core engine: MMA tiles (128 outputs each) per warp, 1, 2 or 3;
     * a product's tiles are spread over the warps of one CTA */
    SNT_OPT_MMA_TILES = 6,
    /* elements each lane group of the R/3 kernel runs at once, 1 or 2 (two
     * independent divstep chains per lane, sharing the shuffles) */
    SNT_OPT_R3_KPT = 7,
    /* tensor-core engine: at most this many warps share one tile's sum on
     * narrow tree levels (1, 2 or 4; 2 from 256 products down, 4 from 64) */
    SNT_OPT_MMA_KSPLIT = 8,
    /* Montgomery's trick over a forest: at most this many equal subtrees
     * (powers of two, 1 .. 1024), each with its own root inversion, all roots
     * inverted in one launch; the tree's narrowest, latency-bound levels are
     * traded for parallel root inversions.  The count used is the largest
     * power of two not above the value that divides B (same bytes for any
     * choice: inverses are unique). */
    SNT_OPT_ROOTS = 9,
    /* R/3 inverses of g: 0 per key by bit-sliced divsteps (which also decide
     * invertibility); 1 the paper's batch path (Sec. 3.1.1): every g is
     * tested invertible by its remainders modulo the irreducible factors of
     * x^p - x - 1 over F_3 (and redrawn until it is), then all are inverted
     * with Montgomery's trick in R/3 (tensor-core product forest, one
     * jump-divstep inversion per subtree); 2 the same forest on the first
     * draws at once, invertibility read off each subtree's root (a product
     * is invertible iff every factor is), a failed subtree redone per key */
    SNT_OPT_R3_MODE = 10,
    /* 1 (default): the tensor-core batch path forms h from the inverses of
     * the tree's level-1 nodes, h_L = 3 inv(P) (g_L f_R) for P = (3f_L)(3f_R),
     * instead of inverting every leaf and then multiplying by g (one small
     * and one half-cost product per key instead of two general ones; p = 653
     * and 761 only: for 857 the limb sums could reach 2^24 and the option is
     * ignored); 0: the leaf level of the down-sweep, then h = g (3f)^-1.
     * Same bytes either way. */
    SNT_OPT_FUSE_LEAF = 11,
    /* R/q inversions of snt_keygen_perkey (one per key): 1 (default) jump
     * divsteps, the kernel of the tree's root inversions (chunks of 31 steps
     * on the low coefficients, the chunk's transition matrix applied to the
     * whole state on the tensor cores); 0 the step-at-a-time kernel (one
     * divstep of the whole state per CTA barrier).  Same bytes either way. */
    SNT_OPT_PERKEY_INV = 12,
    /* 1 (default), 2 or 4: batch keygen splits its forest's subtrees into
     * that many groups of consecutive keys and runs each group from its
     * up-sweep to its pk hash on a stream of its own, so that one group's
     * latency-bound root inversions overlap another group's wide tree levels
     * (tensor-core or transform engine; ignored unless the forest's subtree
     * count is a multiple of it).  Same products, same bytes. */
    SNT_OPT_PARTS = 13,
    /* 1 (default) or 0: launch the kernels of each stream's chain with
     * programmatic stream serialization, so that a kernel's CTAs are
     * scheduled while its predecessor's last wave runs and start the moment
     * it completes (each such kernel waits for its predecessor's completion
     * before its first memory access); 0 launches them plainly.  Same bytes
     * either way; a ragged graph is captured again when it changes. */
    SNT_OPT_PDL = 14,
    /* 0 (default) or a power of two in [1, 1024]: subtrees of the R/3
     * forest of R/3 modes 1 and 2 (0: as many as the R/q forest,
     * SNT_OPT_ROOTS).  The R/3 work runs beside the R/q chain, so a forest of
     * few subtrees (few latency-bound R/3 root inversions holding SMs) can
     * pair with an R/q forest of many.  Same bytes. */
    SNT_OPT_R3_ROOTS = 15
} snt_option;

snt_status snt_ctx_set_option(snt_ctx *ctx, int option, int value);
snt_status snt_ctx_get_option(snt_ctx *ctx, int option, int *value);

/* Autotuner: times batch keygen of B keys of parameter set P on this GPU
 * (CUDA events around calls issued back to back: a warm-up call, then the
 * best of two rounds of two calls) under each candidate layout, times the
 * eight fastest again (the best of two rounds of six calls after a warm-up
 * round), and keeps the fastest of those for every later keygen call of
 * this context with the
 * same P and ceil(log2 B) (and for the ragged call's parameter sets whose
 * largest batch falls in that bucket); it overrides the snt_ctx_set_option
 * values there.  Before each timed call, when the context's scratch has
 * 160 MiB to spare beyond the call's own, a memset of them evicts the L2
 * (outside the call's timed span).  Candidates: R/3 lanes (4, 8, 32) x R/3
 * overlap (0 .. 3) x
 * { tensor-core engine (1, and each of its candidates again as 3) with 1 or
 * 2 MMA tiles per warp, forests of 1, 4, 8, 16, 32, 64, 128 or 256 subtrees
 * (SNT_OPT_ROOTS) and R/3 mode 0, 1 or 2 (modes 1 and 2 also with an R/3
 * forest of 1 or 4 subtrees, SNT_OPT_R3_ROOTS); CUDA-core
 * Toeplitz engine with tree split 4 or 8; transform multiplier (engine 2)
 * with forests of 1, 16, 64 or 128 subtrees and R/3 mode 0 or 2; the
 * tensor-core engine in 2 or 4 pipelined parts (SNT_OPT_PARTS) with forests
 * of 16 .. 256 } (some combinations pruned; one R/3 element per lane group).
 * Synchronous; uses the context's scratch (B must fit the budget).
 * choice (optional, 8 ints): lanes, split, overlap, engine, tiles, kpt, roots,
 * r3 mode. */
snt_status snt_autotune_ex(snt_ctx *ctx, int P, size_t B, int *choice);

/* The layouts the autotuner kept for (P, ceil(log2 B)) on this context:
 * out[0 .. min(n, 10)) = lanes, split, overlap, engine, tiles, kpt, roots,
 * r3 mode, parts, R/3 roots (0: as roots) (all zero if it has not run for
 * that bucket). */
snt_status snt_ctx_tuned(snt_ctx *ctx, int P, size_t B, int *out, int n);

/* snt_autotune_ex returning lanes, split and overlap only. */
snt_status snt_autotune(snt_ctx *ctx, int P, size_t B, int *lanes_out, int *split_out,
                        int *overlap_out);

/* ---- Tracing ---- */

/* Phases reported by snt_ctx_phase_times, in this order: sampling of f, the
 * leaves 3f and g's first draw; the R/3 inversions with any further draws of
 * g (auxiliary stream); tree up-sweep (per-key path: all per-key R/q
 * inversions); root inversion; down-sweep; h = g/(3f) with Rq_encode; SHA-512
 * of the public keys; whole call (main stream, start to end); the wait for
 * the R/3 inversions at the end of the call with the fix-up of resampled
 * keys. */
#define SNT_NPHASES 9

/* Turn per-phase CUDA events on (on != 0) or off for later keygen calls. */
snt_status snt_ctx_set_timing(snt_ctx *ctx, int on);

/* Waits for the last keygen call issued with timing on and writes its phase
 * durations in milliseconds to ms[0 .. SNT_NPHASES). n >= SNT_NPHASES. */
snt_status snt_ctx_phase_times(snt_ctx *ctx, float *ms, int n);

/* ---- Measurement utility (not part of key generation) ---- */

/* Measures the device's integer-pipe throughput with a register-resident
 * stream of independent instructions: kind 0 = LOP3 (3-input logic, the
 * bit-sliced R/3 work), kind 1 = IMAD (32-bit multiply-add, the R/q
 * products), kind 2 = DP4A (4-way 8-bit dot product with 32-bit accumulate),
 * kind 3 = IMAD and LOP3 alternating (both pipes' combined issue rate),
 * kind 4 = PRMT (byte permute), kind 5 = SHF (funnel shift), kind 6 = DP4A
 * and PRMT alternating; kinds 7 and 8 are warp-level tensor MMA streams
 * (m16n8k16 f16 -> f32 and m16n8k32 s8 -> s32) and report multiply-adds
 * per second instead of instructions.
 * Writes instructions per second (summed over all SMs) to *ops_per_s and the
 * SM count to *sms.  Synchronous; uses no scratch. */
snt_status snt_measure_int_peak(int device, int kind, double *ops_per_s, int *sms);

/* Measures the 5th-generation tensor-core MMA (tcgen05.mma kind::f16: f16
 * operands from shared memory, f32 accumulator in tensor memory) at M = 128,
 * K = 16 and N = n (16, 32, 64, 128 or 256): ctas_per_sm (1, 2 or 4; at most
 * 512 tensor-memory columns per SM, max(32, n) per CTA) CTAs per SM, each
 * with one thread issuing back-to-back MMAs into its accumulator, the result
 * checked against its closed form.  Writes multiply-adds per second (all SMs) to *macs_per_s and
 * the SM count to *sms.  The rate at small N bounds what a tcgen05 form of
 * the R/q Toeplitz products could reach (no calls of key generation use
 * it).  Returns SNT_EINTERNAL if the accumulator is wrong, SNT_ETIMEOUT if
 * the MMAs did not complete in about two seconds.  Synchronous. */
snt_status snt_measure_tc05(int device, int n, int ctas_per_sm, double *macs_per_s, int *sms);

/* One-line description of the last error on this host thread. */
const char *snt_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* SNTRUP_GB300_H */
