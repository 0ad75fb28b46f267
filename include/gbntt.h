/*
 * gbntt.h -- C ABI of the GB300 modular NTT library (libgbntt.so).
 *
 * Exact number-theoretic transforms over F_p, p = k 2^l + 1 a word-size
 * prime, and the products built on them, after van der Hoeven, Lecerf and
 * Quintin, "Modular SIMD arithmetic in Mathemagix" (2014):
 *   - the transform FFT_w / TFT_w of Section 5.1 (Algorithm 1),
 *   - the polynomial product over Z/pZ of Section 5.2,
 *   - the three-prime integer product of Section 5.3.
 *
 * Conventions for every call:
 *   - Residues are stored as their representative in {0, ..., p-1}
 *     (Section 2).  Words are uint32_t when p < 2^32, uint64_t when
 *     2^32 <= p < 2^62; a plan reports which (word_bytes).
 *   - Pointers named d_* are caller-owned DEVICE memory; h_* are host
 *     memory.  The library never frees or keeps caller buffers.  Inputs are
 *     never modified, except by the in-place transforms.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device calls are asynchronous on that stream; an OK return
 *     means the work was enqueued.  Errors detected on the host return
 *     before anything is enqueued.
 *   - Every call returns an int status: NTT_OK (0) or an NTT_ERR_* code;
 *     ntt_status_str() names it and ntt_last_error() gives details for the
 *     calling thread.
 *   - A plan is immutable after creation and may be shared across threads
 *     and streams.  Hot calls allocate nothing: calls that need scratch
 *     memory take a caller workspace whose size the *_workspace_size
 *     queries return.
 */
#ifndef GBNTT_H
#define GBNTT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum ntt_status {
    NTT_OK = 0,
    NTT_ERR_ARG = 1,          /* null pointer, bad flag or enum value */
    NTT_ERR_MODULUS = 2,      /* p even, p < 3, p >= 2^62, or 16 does not divide p-1 */
    NTT_ERR_NOT_PRIME = 3,    /* p is not prime */
    NTT_ERR_NO_ROOT = 4,      /* 2^log2n does not divide p - 1 */
    NTT_ERR_SIZE = 5,         /* sizes exceed what the plan supports */
    NTT_ERR_RANGE = 6,        /* an input residue is >= p (NTT_FLAG_CHECK only) */
    NTT_ERR_OOM = 7,          /* device or host allocation failed */
    NTT_ERR_TIMEOUT = 8,      /* a bounded device wait expired */
    NTT_ERR_CUDA = 9,         /* a CUDA runtime call failed */
    NTT_ERR_WORKSPACE = 10,   /* workspace missing or too small */
    NTT_ERR_UNSUPPORTED = 11  /* valid request this build does not implement */
};

/* Plan creation flags. */
#define NTT_FLAG_PLAIN 0x1u   /* also build the tables of the one-launch-per-stage schedule */
#define NTT_FLAG_CHECK 0x2u   /* validate input ranges on the host side of each call */
#define NTT_FLAG_FP64 0x4u    /* residues held as IEEE doubles, products by Function 16
                                 (Section 3.3); needs p < 2^50; transforms and products only */

/* Schedules for polymul_mod_p_batch. */
#define NTT_SCHED_FUSED 0u    /* Algorithm 1 passes fused in shared memory */
#define NTT_SCHED_PLAIN 1u    /* one kernel launch per radix-2 stage (baseline) */

/* Modular-product variants for ntt_modmul_vec (Sections 2.2, 2.3, 3.3). */
#define NTT_MM_BARRETT 0u     /* Function 6 on the full product x*y, Table 3 parameters */
#define NTT_MM_SHOUP 1u       /* Function 8: y fixed, companion psi = floor(2^n y / p) */
#define NTT_MM_MONTGOMERY 2u  /* Function 13 on x~ y~ (inputs in Montgomery form) */
#define NTT_MM_FMA 3u         /* Function 16 over IEEE double, p < 2^50 */
#define NTT_MM_MONT_FIXED 4u  /* Remark 8: y fixed, companion phi; kernels' twiddle product */
#define NTT_MM_MONT_PRODUCT 5u /* the kernels' general (pointwise) product: x y 2^-n rem p, scaled back */
#define NTT_MM_ADD 6u         /* the kernels' modular sum x + y rem p (Section 2.1) */
#define NTT_MM_SUB 7u         /* the kernels' modular difference x - y rem p */
#define NTT_MM_MONT_FIXED_W 8u   /* n = 32: Remark 8's product from the 64-bit product x y~ (no
                                    companion), borrow-mask tail; the row pass's twiddle product */
#define NTT_MM_MONT_PRODUCT_W 9u /* n = 32: the row pass's pointwise product (same forms), scaled back */

typedef struct ntt_plan ntt_plan;

typedef struct ntt_plan_info {
    uint64_t p;           /* the modulus */
    uint64_t g;           /* least generator of F_p^* */
    uint64_t omega;       /* primitive n-th root used: g^((p-1)/n) */
    uint64_t omega_inv;   /* omega^-1 rem p */
    uint64_t n_inv;       /* n^-1 rem p */
    uint32_t log2n;       /* n = 2^log2n */
    uint32_t word_bytes;  /* 4 or 8 */
    uint32_t v2;          /* largest l with 2^l | p - 1 */
    uint32_t tile_max_log;/* largest log2n transformed by one thread block */
} ntt_plan_info;

/* ---- host-only planning (no GPU needed) -------------------------------- */

/* The index-th (0-based) prime p = k 2^min_l + 1 with 2^(bits-1) < p < 2^bits,
 * by ascending k (Section 1: moduli p = k 2^l + 1 with l large).
 * bits in [3, 63], min_l < bits - 1.  Writes *p_out.
 * NTT_ERR_ARG on bad arguments, NTT_ERR_SIZE if the window holds fewer
 * than index+1 such primes. */
int ntt_find_prime(unsigned bits, unsigned min_l, unsigned index, uint64_t* p_out);

/* The least generator g of F_p^* and omega = g^((p-1)/2^log2n), the
 * primitive 2^log2n-th root of unity every transform of this library uses
 * (Section 5.1 requires a primitive n-th root; this fixes which one).
 * NTT_ERR_NOT_PRIME, NTT_ERR_NO_ROOT as for ntt_plan_create. */
int ntt_root_of_unity(uint64_t p, unsigned log2n, uint64_t* g_out, uint64_t* omega_out);

/* Host computation of the fixed-multiplicand companions for ntt_modmul_vec,
 * for words of n = 8 * word_bytes bits: kind NTT_MM_SHOUP: out[i] =
 * floor(2^n y[i] / p) (Function 8's psi); NTT_MM_MONT_FIXED (n = 32 only):
 * out[i] = (y[i] 2^32 rem p) p^-1 rem 2^32 (Remark 8's companion of the
 * Montgomery form).  Host buffers; y[i] are reduced mod p first. */
int ntt_fixed_companion(uint64_t p, unsigned kind, unsigned word_bytes, const uint64_t* h_y,
                        uint64_t* h_out, size_t n);

/* ---- plans ------------------------------------------------------------- */

/* Create a plan for transforms of length n = 2^log2n over F_p on the
 * current CUDA device: checks p (prime, odd, < 2^62, 16 | p-1) and
 * 2^log2n | p-1, builds the root-of-unity tables on the host (Section 5.1:
 * all powers precomputed and cached) and copies them to the device once.
 * For log2n = 17 .. 24 the plan also owns a 2^16-point plan of the same
 * modulus and a table of 2n twiddles (the transform is Algorithm 1 over
 * 2^16-point rows).  1 <= log2n <= 24.  flags: NTT_FLAG_*.  The plan owns
 * its device tables; free it with ntt_plan_destroy.  Errors: NTT_ERR_ARG,
 * NTT_ERR_MODULUS, NTT_ERR_NOT_PRIME, NTT_ERR_NO_ROOT, NTT_ERR_SIZE,
 * NTT_ERR_OOM, NTT_ERR_CUDA, NTT_ERR_UNSUPPORTED (NTT_FLAG_FP64 with
 * NTT_FLAG_PLAIN). */
int ntt_plan_create(uint64_t p, unsigned log2n, unsigned flags, ntt_plan** out);

/* Free the plan and its device tables (synchronises the plan's device). */
int ntt_plan_destroy(ntt_plan* plan);

/* Fill *out with the plan's parameters. */
int ntt_plan_get_info(const ntt_plan* plan, ntt_plan_info* out);

/* ---- transforms ---------------------------------------------------------- */

/* In-place forward transform of `batch` vectors of n words stored back to
 * back at d_data: vector v becomes TFT_omega with l = n (Section 5.1),
 * i.e. word i holds A(omega^[i]) where [i] mirrors the log2n bits of i.
 * Inputs must be residues < p (NTT_FLAG_FP64 plans: doubles holding them).
 * For n = 2^16 .. 2^24 the fast passes need d_data 16-byte aligned; data
 * that is only word-aligned gets the same result from slower passes. */
int ntt_forward(const ntt_plan* plan, void* d_data, size_t batch, void* stream);

/* In-place inverse: consumes the bit-mirrored order ntt_forward produces and
 * returns natural order scaled by n^-1, so ntt_inverse(ntt_forward(a)) = a
 * (the inverse of Algorithm 1, text after Proposition 15). */
int ntt_inverse(const ntt_plan* plan, void* d_data, size_t batch, void* stream);

/* ---- polynomial products over Z/pZ (Section 5.2) ---------------------- */

/* Workspace bytes polymul_mod_p_batch needs for `batch` products with this
 * plan and schedule (0 when none is needed). */
size_t polymul_workspace_size(const ntt_plan* plan, size_t batch, unsigned schedule);

/* c = a * b over Z/pZ for `batch` independent pairs: a is batch x na words,
 * b is batch x nb words, c is batch x (na + nb - 1) words, all row-major and
 * back to back.  Requires 1 <= na, nb and na + nb - 1 <= n: the product is
 * the size-n cyclic convolution of the zero-padded operands, which equals the
 * linear product when no coefficient wraps.  Two forward transforms, the
 * pointwise product and one inverse transform (Section 5.2).  From n = 2^9
 * on, the transforms are truncated (TFT, Section 5.1) to the blocks of
 * n/16 positions (rows of 2^16 words above 2^16 points) that the na + nb - 1
 * output words need, wherever that measured faster; this changes nothing in
 * c.  schedule:
 * NTT_SCHED_FUSED or NTT_SCHED_PLAIN (the latter needs NTT_FLAG_PLAIN).
 * d_ws: at least polymul_workspace_size bytes, 256-byte aligned (may be
 * NULL when that size is 0). */
int polymul_mod_p_batch(const ntt_plan* plan, const void* d_a, size_t na,
                        const void* d_b, size_t nb, size_t batch, void* d_c,
                        unsigned schedule, void* d_ws, size_t ws_bytes, void* stream);

/* Device staging bytes polymul_mod_p_batch_host needs for chunks of `chunk`
 * products of na x nb words: three sets of one chunk's operands and result,
 * plus the workspace of one chunk (0 on bad arguments). */
size_t polymul_host_stage_size(const ntt_plan* plan, size_t na, size_t nb, size_t chunk);

/* polymul_mod_p_batch (fused schedule; the products of Section 5.2) for
 * operands and results in HOST memory: h_a is batch x na words, h_b batch x
 * nb words, h_c receives batch x (na + nb - 1) words, laid out as for
 * polymul_mod_p_batch.  The batch is cut into chunks of at most `chunk`
 * products (a long batch starts and ends with chunk/4 and chunk/2);
 * the upload of one chunk, the product of the previous one (on `stream`)
 * and the download of the one before run concurrently, through two library
 * copy streams per device (created on the first call on that device and
 * kept until exit).  Overlap needs page-locked host memory (cudaHostAlloc
 * or cudaHostRegister); pageable memory gives the same result, slower.
 * d_stage: caller-owned device memory of at least polymul_host_stage_size
 * bytes for this chunk, 256-byte aligned; it and the host buffers are in
 * use until the call's work on `stream` completes, which is also when h_c
 * holds the result.  The plan's device must be current.  Errors as for
 * polymul_mod_p_batch; NTT_ERR_WORKSPACE for a missing or short d_stage.
 * Argument errors return before anything is enqueued; a CUDA runtime error
 * while enqueueing (NTT_ERR_CUDA) can leave earlier chunks enqueued. */
int polymul_mod_p_batch_host(const ntt_plan* plan, const void* h_a, size_t na, const void* h_b,
                             size_t nb, size_t batch, void* h_c, size_t chunk, void* d_stage,
                             size_t stage_bytes, void* stream);

/* The single-product form of polymul_mod_p_batch (fused schedule). */
int polymul_mod_p(const ntt_plan* plan, const void* d_a, size_t na, const void* d_b,
                  size_t nb, void* d_c, void* d_ws, size_t ws_bytes, void* stream);

/* polymul_mod_p_batch with the fused schedule for callers that cannot
 * allocate device memory when they need a product: hosts that own all
 * device memory through their own allocator or a budget fixed at start-up,
 * and latency-critical loops that cannot take an allocation's implicit
 * synchronisation or the risk of its failing mid-run.  The paper has no
 * counterpart (its products run on the CPU).  Operands and output are as
 * for polymul_mod_p_batch; the scratch space the larger transforms need
 * comes from a fixed 32 MiB array inside the library (held on every GPU
 * that loads the library until the process exits), so this call allocates
 * nothing.  Products needing more scratch than that (2 n word_bytes per
 * product when n > 2^tile_max_log: at most 64 products of n = 2^16 with
 * 32-bit words, 32 with 64-bit words) return NTT_ERR_WORKSPACE.  The first
 * call on each device (and the first after that device's context changes,
 * e.g. after cudaDeviceReset) looks up the array's address with
 * cudaGetSymbolAddress; make that first call before any stream capture.
 * Every call shares the one array, which keeps the last call's contents:
 * calls whose work overlaps on the GPU race and must be serialised by the
 * caller.  A plan created with NTT_FLAG_CHECK copies the operands to the
 * host and synchronises the stream on every call, as polymul_mod_p_batch
 * does.  The plan's device must be current. */
int polymul_mod_p_batch_static(const ntt_plan* plan, const void* d_a, size_t na,
                               const void* d_b, size_t nb, size_t batch, void* d_c,
                               void* stream);

/* ---- polynomial matrix products (Section 5.2) ---------------------------- */

/* Workspace bytes for polymat_mul with this plan and n x n matrices. */
size_t polymat_workspace_size(const ntt_plan* plan, unsigned n);

/* C = A B for n x n matrices of polynomials over Z/pZ of degree < d:
 * transforms of length 2^log2n of every entry, an n x n matrix product over
 * F_p at every frequency, inverse transforms of the n^2 entries of C
 * (Section 5.2, the polynomial matrix product).  A, B: entry (i, j) at word
 * (i n + j) d, d words each; C: entry (i, j) at (i n + j)(2d - 1).  Needs
 * 2d - 1 <= 2^log2n and 1 <= n <= 1024.  Workspace: polymat_workspace_size. */
int polymat_mul(const ntt_plan* plan, const void* d_A, const void* d_B, unsigned n, size_t d,
                void* d_C, void* d_ws, size_t ws_bytes, void* stream);

/* ---- uneven batches with mixed moduli ------------------------------------ */

/* One product of an uneven batch: operands a[a_off .. a_off+na) and
 * b[b_off .. b_off+nb), output c[c_off .. c_off+na+nb-1), offsets in words
 * into the run's flat buffers; `prime` indexes the plan's modulus list. */
typedef struct polymul_desc {
    uint64_t a_off, b_off, c_off;
    uint32_t na, nb;
    uint32_t prime;
    uint32_t reserved;
} polymul_desc;

/* Run modes of polymul_batch_run. */
#define NTT_BATCH_DIRECT 0u   /* every launch on the caller's stream, in order */
#define NTT_BATCH_STREAMS 1u  /* buckets spread over internal streams, joined back */
#define NTT_BATCH_GRAPH 2u    /* the STREAMS work captured once into a CUDA graph, replayed */

typedef struct polymul_batch_plan polymul_batch_plan;

/* Plan `count` products of uneven lengths over up to 64 moduli (all below
 * 2^32, or all in [2^32, 2^62)).  Host descriptors are read once.  Each
 * product's transform length is the least 2^k >= na + nb - 1.  Products
 * with 2^k within one thread block become items of a persistent kernel
 * that takes them from a ticket counter (largest first, up to 16 equal-size
 * equal-modulus products per item, items truncated to the blocks their
 * longest output needs); longer products are grouped by (modulus, k, and
 * below 2^16 points whether truncation pays) and run as the fused three-pass
 * schedule, each product truncated to its own output length.  Allocates the
 * transform plans and the device descriptor tables (not a hot call).
 * flags: reserved, pass 0. */
int polymul_batch_plan_create(const uint64_t* primes, unsigned nprimes, const polymul_desc* h_desc,
                              size_t count, unsigned flags, polymul_batch_plan** out);
int polymul_batch_plan_destroy(polymul_batch_plan* plan);

/* Workspace bytes polymul_batch_run needs (the ticket counter and the
 * long products' transformed operands). */
size_t polymul_batch_workspace_size(const polymul_batch_plan* plan);

/* Every product of the plan, reading d_a / d_b and writing d_c at the
 * descriptors' offsets (device buffers, words of the plan's size).  mode:
 * NTT_BATCH_*.  In NTT_BATCH_GRAPH mode the first run with a given set of
 * (d_a, d_b, d_c, d_ws) captures the work into a CUDA graph (allocating the
 * graph); later runs with the same pointers only launch it.  Not thread-safe
 * for one plan. */
int polymul_batch_run(polymul_batch_plan* plan, const void* d_a, const void* d_b, void* d_c,
                      void* d_ws, size_t ws_bytes, unsigned mode, void* stream);

/* ---- serving loop ------------------------------------------------------------ */

/* Request kinds and flags for ntt_server_submit. */
#define NTT_REQ_INTMUL 0u     /* integer product, 32-bit limbs (Section 5.3) */
#define NTT_REQ_POLYMUL 1u    /* polynomial product over Z/P_iZ, 64-bit words (Section 5.2) */
#define NTT_REQ_DEVICE 0x1u   /* a, b, c are device buffers: no copies, no operand memory */

typedef struct ntt_server_config {
    size_t max_limbs;   /* largest operand (limbs, or words for polynomial products) */
    size_t mem_bytes;   /* device arena for operands, outputs and scratch */
    unsigned slots;     /* requests in flight at once (one CUDA stream each) */
    unsigned reserved;
} ntt_server_config;

typedef struct ntt_server ntt_server;

/* Start a server on the current device: builds the transform tables of the
 * three 62-bit primes for every length up to max_limbs, allocates the arena
 * and `slots` streams, and starts the scheduler thread.  (The paper has no
 * serving loop; its products run one at a time.) */
int ntt_server_create(const ntt_server_config* cfg, ntt_server** out);

/* Queue a product: c = a * b with a of na and b of nb elements.  For
 * NTT_REQ_INTMUL, c receives na + nb limbs; for NTT_REQ_POLYMUL, c receives
 * na + nb - 1 words reduced modulo P_prime (prime in 0..2).  Host buffers
 * (pinned for asynchronous copies) unless NTT_REQ_DEVICE; they must stay
 * valid until the request completes.  Requests are admitted in arrival
 * order when a slot and arena memory are free.  *id_out identifies it.
 * NTT_ERR_SIZE / NTT_ERR_OOM if it can never fit. */
int ntt_server_submit(ntt_server* server, unsigned kind, unsigned prime, const void* a, size_t na,
                      const void* b, size_t nb, void* c, unsigned flags, uint64_t* id_out);

/* *state: 0 pending, 1 running, 2 done, 3 failed; *latency_ms (done or
 * failed only): submission to completion of the result copy, host clock.
 * Returns the request's error status once it failed. */
int ntt_server_poll(ntt_server* server, uint64_t id, int* state, double* latency_ms);

/* Wait up to timeout_ms for the request; NTT_ERR_TIMEOUT if it is not done. */
int ntt_server_wait(ntt_server* server, uint64_t id, int timeout_ms, double* latency_ms);

/* Forget a finished request. */
int ntt_server_release(ntt_server* server, uint64_t id);

int ntt_server_stats(ntt_server* server, uint64_t* completed, uint64_t* pending, uint64_t* running,
                     uint64_t* peak_inflight);

/* Stop the scheduler, wait for work in flight, free everything. */
int ntt_server_destroy(ntt_server* server);

/* ---- launch-shape autotuning ------------------------------------------------ */

/* Time the candidate launch shapes of the fused product for this plan's
 * transform length on `batch` products of length n/2 (temporary device
 * buffers are allocated) and keep the fastest in the process-wide shape
 * table used by every later launch of that (word size, log2 n).  Writes the
 * best time in ms to *best_ms when non-null.  Synchronous. */
int ntt_autotune(const ntt_plan* plan, size_t batch, void* stream, float* best_ms);
/* The shape currently used for (word_bytes, log2n): products per block,
 * columns per block and rows per block, each as log2.  For n = 2^16 .. 2^24
 * above the one-block limit, logw = 0 (the default) selects the direct
 * kernels, whose block shape is fixed (lrpc is then ignored); at n = 2^16,
 * lppc = 1 makes them bring zero-half operand tiles in by TMA.  The
 * autotuner never picks that shape (a block whose bounded TMA waits both
 * expire would return with its copy still in flight); it is set only
 * through ntt_tune_import. */
int ntt_tune_get(unsigned word_bytes, unsigned log2n, int* lppc, int* logw, int* lrpc);
/* Forget every tuned or imported shape (back to the defaults). */
int ntt_tune_reset(void);
/* Text form of the shape table ("word_bytes log2n lppc logw lrpc" lines):
 * export into buf (cap bytes; *len receives the length; buf may be NULL to
 * query it) and import such text back. */
int ntt_tune_export(char* buf, size_t cap, size_t* len);
int ntt_tune_import(const char* text);

/* ---- integer products (Section 5.3) ------------------------------------- */

typedef struct intmul_plan intmul_plan;

/* Plan for products of integers of up to max_limbs 32-bit limbs each: the
 * three primes P1 < P2 < P3 = the first three k 2^40 + 1 above 2^61
 * (ntt_find_prime(62, 40, i)), a transform plan per prime for every length
 * 2^1 .. 2^k the largest product needs, and the Garner constants.  Builds
 * all tables up front (this call allocates; intmul_crt does not).
 * NTT_ERR_SIZE if a product would need transforms above 2^24. */
int intmul_plan_create(size_t max_limbs, intmul_plan** out);
int intmul_plan_destroy(intmul_plan* plan);

/* Workspace bytes intmul_crt needs for operands of na and nb limbs. */
size_t intmul_workspace_size(const intmul_plan* plan, size_t na, size_t nb);

/* c = a * b for non-negative integers in little-endian 32-bit limbs:
 * a has na >= 1 limbs, b has nb >= 1, c receives exactly na + nb limbs.
 * Kronecker segmentation into chunks of Section 5.3's size h, the largest
 * h <= 96 with 2 h + bitlength(min(da, db)) <= 183 (da, db the chunk counts;
 * 80 to 91 bits at 2^14 .. 2^28-bit operands), the product modulo each of
 * the three primes (two forward transforms, pointwise product, inverse),
 * Garner reconstruction of every coefficient (exact: coefficients are below
 * 2^183 < P1 P2 P3) and carry propagation.  d_ws: at least
 * intmul_workspace_size bytes, 256-byte aligned.  Asynchronous on stream. */
int intmul_crt(const intmul_plan* plan, const uint32_t* d_a, size_t na, const uint32_t* d_b,
               size_t nb, uint32_t* d_c, void* d_ws, size_t ws_bytes, void* stream);

/* Workspace bytes intmat_mul needs for n x n matrices of na- and nb-limb entries. */
size_t intmat_workspace_size(const intmul_plan* plan, unsigned n, size_t na, size_t nb);

/* C = A B for n x n matrices of non-negative integers (Section 5.3's
 * integer matrix product by modular transforms): every entry of A has na
 * 32-bit limbs, every entry of B nb limbs; entry (i, j) of C receives
 * na + nb + 1 limbs (a sum of n products of na + nb limbs each needs one
 * limb more).  Entries are cut into 64-bit chunks, the polynomial matrix
 * product is taken modulo each of the three primes (polymat_mul's method),
 * and every coefficient (a sum of n d products below 2^128, d = the larger
 * chunk count) is rebuilt by Garner's CRT and carried.  A: entry (i, j) at
 * limb (i n + j) na; B likewise with nb; C with na + nb + 1.  1 <= n <= 255.
 * The plan must cover transforms of length >= 2d - 1. */
int intmat_mul(const intmul_plan* plan, const uint32_t* d_A, size_t na, const uint32_t* d_B, size_t nb,
               unsigned n, uint32_t* d_C, void* d_ws, size_t ws_bytes, void* stream);

/* ---- element-wise modular operations (Sections 2.1-2.3, 3.3) ----------- */

/* z[i] = x[i] * y[i] rem p with the reduction `kind` (NTT_MM_*; kinds
 * NTT_MM_ADD / NTT_MM_SUB give x[i] + y[i] and x[i] - y[i] rem p), on uint64
 * device arrays of residues < p.  word_bytes selects the 32- or 64-bit
 * implementation (4 needs p < 2^32).  NTT_MM_SHOUP / NTT_MM_MONT_FIXED read
 * the companions d_yc (from ntt_fixed_companion); other kinds ignore it.
 * NTT_MM_MONTGOMERY converts x, y to Montgomery form, multiplies with
 * Function 13 and converts back.  NTT_MM_FMA needs p < 2^50.
 * NTT_MM_MONT_FIXED_W and NTT_MM_MONT_PRODUCT_W need word_bytes = 4. */
int ntt_modmul_vec(uint64_t p, unsigned kind, unsigned word_bytes, const uint64_t* d_x,
                   const uint64_t* d_y, const uint64_t* d_yc, uint64_t* d_z, size_t n,
                   void* stream);

/* Throughput of one reduction variant (kinds NTT_MM_BARRETT .. NTT_MM_MONT_FIXED)
 * on register-resident operands: every GPU thread runs 4 independent chains
 * of `iters` dependent products x <- x y rem p by a fixed y.  Writes modular
 * products per second; synchronous; allocates a small buffer.  This is the
 * measurement behind Sections 2-3's comparison of reductions, taken on the
 * GPU (Tables 5-8 and 10 time them on one CPU core). */
int ntt_modmul_rate(uint64_t p, unsigned kind, unsigned word_bytes, int iters, double* products_per_s);

/* ---- diagnostics --------------------------------------------------------- */

/* NTT_OK, or NTT_ERR_TIMEOUT when a kernel's bounded wait for a tensor-
 * memory-accelerator (TMA) copy on the current device ran out since the
 * last call (the kernel then returned without writing its results; the flag
 * is cleared by this call).  Synchronous (reads one device word). */
int ntt_device_status(void);

/* Launch profiling (the paper has no counterpart; it reports CPU user time
 * per transform, Section 5.1).  After ntt_profile_begin(), every library
 * call records a CUDA event on its own stream after each kernel it
 * enqueues.  ntt_profile_end() stops recording, waits for the last event
 * and reports, for each kernel launched since begin (at most max_kernels),
 * its device time in ms and its static name; *count gets the number of
 * kernels.  Process-wide; not for concurrent use from several threads. */
int ntt_profile_begin(void);
int ntt_profile_end(int max_kernels, float* ms_out, const char** names_out, int* count);

/* Integer-pipe throughput probe: `blocks` x `threads` threads run
 * independent chains of 32-bit multiply-adds (kind 0), of adds/xors
 * (kind 1), of both interleaved 1:1 (kind 2: the issue ceiling of integer
 * work split evenly over the multiply-add and ALU pipes, the roof of the
 * transform kernels), or of 32 x 32 -> 64-bit multiply-adds (kind 3),
 * 64 * iters operations each; writes operations per second to *ops_per_s
 * (timed with CUDA events on `stream`; synchronous).  Not part of the
 * paper: a measurement of the machine.  Allocates a small device buffer. */
int ntt_int_probe(unsigned kind, int blocks, int threads, int iters, void* stream,
                  double* ops_per_s);

const char* ntt_status_str(int status);
/* Details of the last error on the calling thread ("" if none). */
const char* ntt_last_error(void);
/* Library version string. */
const char* ntt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBNTT_H */
