/*
 * moma.h -- C ABI of the GB300 (sm_103a) multi-word modular arithmetic library.
 *
 * The operations are those of "Code Generation for Cryptographic Kernels using
 * Multi-word Modular Arithmetic on GPU" (Zhang & Franchetti, CGO'25):
 *   - element-wise modular BLAS over Z_q: addmod, submod, mulmod (Sec. 2.1, Eq. 1)
 *     and axpy y' = a*x + y (Sec. 2.3);
 *   - the forward cyclic number theoretic transform y(k) = sum_j x(j) w_n^(jk) mod q
 *     (Sec. 2.3, Eq. ntt) and its inverse;
 *   - the cyclic polynomial product through the transform (Sec. 2.3).
 * Large-modulus arithmetic is broken into 32-bit machine words (Sec. 3, Eq. def_moma).
 *
 * Conventions shared by every call
 * --------------------------------
 * Widths.  bits in {128, 256, 384, 768} (the widths of the workloads), and 64, 512, 1024
 *   (the ends of the paper's width sweep, Sec. 5.4); L = bits/32 limbs of 32 bits.  The
 *   modulus q must be odd and have exactly bits-4 bits (Sec. 5.2: a (k-4)-bit modulus for a
 *   k-bit container, which the Barrett constants of Sec. 3.1 need); otherwise
 *   MOMA_ERR_MODULUS.  Every width is supported by every call, except moma_ntt_fwd_noalloc
 *   (64 to 384 bits).  Full-width moduli (up to all bits of the container) take
 *   moma_ctx_create_full (Montgomery reduction); see there for the calls they support.
 * Layout.  A vector of n residues is limb-major: uint32 v[L][n], limb 0 the least
 *   significant word of each residue (the paper writes words most significant first;
 *   that is notation only).  Plane j of element i is at v[j*n + i].
 * Values.  Inputs must be canonical, 0 <= x < q.  Outputs are canonical.  A
 *   non-canonical input gives an unspecified (but memory-safe) result.
 * Memory.  Vector arguments are device pointers owned by the caller; the library never
 *   frees them.  They must be 4-byte aligned; 16-byte aligned planes (n a multiple of
 *   4 and 16-byte aligned base) take the vectorised path.  Outputs may alias inputs
 *   exactly (out == in); partial overlap is undefined.
 * Streams.  `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *   asynchronous: the return code reports argument, configuration and launch errors
 *   only.  Errors raised on the device (a bounded wait that ran out) are recorded in
 *   the context and returned by moma_ctx_sync_status().
 * Threads.  A context may be used from several host threads; plan creation and the
 *   schedule table (moma_ctx_set_config, and the lookups every call makes) are serialised
 *   inside the context.  Calls that overlap on the device and write the same buffers race,
 *   as with any CUDA kernel.
 */
#ifndef MOMA_H
#define MOMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct moma_ctx moma_ctx;

typedef enum {
  MOMA_OK = 0,
  MOMA_ERR_INVALID_ARG = 1, /* null pointer, bad width, n out of range for the call */
  MOMA_ERR_MODULUS = 2,     /* q even, wrong bit length, or (for the NTT) not prime  */
  MOMA_ERR_SIZE = 3,        /* NTT size not a power of two, > 2^24, or not | q-1     */
  MOMA_ERR_ALIGN = 4,       /* device pointer not 4-byte aligned                     */
  MOMA_ERR_OOM = 5,         /* device or host allocation failed                      */
  MOMA_ERR_CUDA = 6,        /* a CUDA runtime call failed (launch, copy, event)      */
  MOMA_ERR_TIMEOUT = 7,     /* a bounded device-side wait ran out                    */
  MOMA_ERR_BUDGET = 8,      /* a job does not fit the memory budget it was given     */
  MOMA_ERR_UNSUPPORTED = 9  /* valid request the library does not implement          */
} moma_status;

/* Human-readable name of a status code (static string, never NULL). */
const char *moma_status_string(moma_status s);

/* ------------------------------------------------------------------ contexts */

/* Create a context for modulus q (host array of bits/32 limbs, least significant
 * first; bits one of the widths above, else MOMA_ERR_INVALID_ARG).  Precomputes the Barrett constant mu = floor(2^(2B+3)/q), B = bits-4
 * (Sec. 3.1, Eq. mu) and the other per-modulus constants, and uploads them.  Transform
 * plans (twiddle tables) are built lazily per size.  *out receives the context; it is
 * set to NULL on error.  Uses the current CUDA device. */
moma_status moma_ctx_create(const uint32_t *q, int bits, moma_ctx **out);

/* Context for a full-width modulus: q odd, with more than bits-32 and at most `bits` bits
 * (the top limb nonzero, up to a modulus that fills the container), else MOMA_ERR_MODULUS.
 * Sec. 5.2 names Montgomery reduction for such moduli, where the 4 spare bits that the
 * Barrett constants of Sec. 3.1 need are absent.  Products by a constant (twiddles, the axpy
 * scalar, n^-1, kept in Montgomery form internally) are word-serial Montgomery products
 * (R = 2^bits, q' = -q^-1 mod 2^32, 2L^2 + L word products); the element-wise product of two
 * vectors (moma_vec_mulmod) is the double-width product reduced by a word-based Barrett
 * reduction with the (L+1)-limb constant floor(2^(2 bits)/q), or, with engine 4 of
 * moma_config, two Montgomery products (the second by R^2 mod q); sums form their carry word.
 * Inputs and outputs are canonical residues as for moma_ctx_create (no Montgomery form is
 * visible to the caller).  Every call accepts such a context; calls other than
 * moma_vec_mulmod ignore the product engine setting.  In batches their jobs run with the
 * per-call kernels after the persistent launch, like 768-bit jobs. */
moma_status moma_ctx_create_full(const uint32_t *q, int bits, moma_ctx **out);

/* 1 for a context made by moma_ctx_create_full, else 0 (also for NULL). */
int moma_ctx_is_full(const moma_ctx *ctx);

/* Release the context, its plans and device tables.  Safe on NULL.  The caller must
 * ensure no work using the context is still running. */
void moma_ctx_destroy(moma_ctx *ctx);

/* Number of 32-bit limbs L of the context (0 for NULL). */
int moma_ctx_limbs(const moma_ctx *ctx);

/* Bytes of device memory the context holds right now: the twiddle tables of every
 * transform plan built so far (one per size, direction and schedule; about n entries of
 * 2L words per direction) and its status word.  Scratch buffers of calls in flight are not
 * included (they come from the stream-ordered pool and are released by the calls).  For
 * admission control by memory budget.  0 for NULL. */
size_t moma_ctx_device_bytes(const moma_ctx *ctx);

/* Write the primitive n-th root of unity w_n the transforms use (L host limbs):
 * w_n = g^((q-1)/n) with g the smallest integer >= 2 that is a quadratic non-residue
 * mod q (the paper leaves the choice of root open, Sec. 2.3).  n a power of two
 * dividing q-1, 2 <= n <= 2^24. */
moma_status moma_ctx_root(moma_ctx *ctx, size_t n, uint32_t *w_out);

/* Block until all work the context issued is done and return (then clear) the first
 * device-side error recorded since the last call (MOMA_ERR_TIMEOUT), else MOMA_OK. */
moma_status moma_ctx_sync_status(moma_ctx *ctx);

/* Bound, in nanoseconds of GPU global time, of every wait of this context's staged BLAS
 * kernels on a shared-memory stage filled by bulk copies (default 2e9).  A wait that runs
 * out records MOMA_ERR_TIMEOUT (see moma_ctx_sync_status); the kernel waits, bounded again,
 * for its copies still in flight and returns, so it never hangs.  ns 0 is MOMA_ERR_INVALID_ARG. */
moma_status moma_ctx_set_wait_limit(moma_ctx *ctx, uint64_t ns);

/* Test hook: the next staged BLAS launch of this context arms its first CTA's first stage
 * for 16 bytes more than its copies deliver, so that one wait runs out (the copies themselves
 * complete normally).  That launch's results are undefined; moma_ctx_sync_status then
 * reports MOMA_ERR_TIMEOUT. */
moma_status moma_ctx_inject_missing_copy(moma_ctx *ctx);

/* ------------------------------------------------------------------ modular BLAS */

/* c[i] = a[i] + b[i] mod q, i < n (Sec. 2.1 Eq. 1 and Eq. saddmod).  n may be 0. */
moma_status moma_vec_addmod(moma_ctx *ctx, size_t n, const uint32_t *a, const uint32_t *b,
                            uint32_t *c, void *stream);

/* c[i] = a[i] - b[i] mod q (Sec. 2.1 Eq. 1 and Eq. ssubmod). */
moma_status moma_vec_submod(moma_ctx *ctx, size_t n, const uint32_t *a, const uint32_t *b,
                            uint32_t *c, void *stream);

/* c[i] = a[i] * b[i] mod q by multi-word Barrett reduction (Sec. 3.1 Eq. barrett and
 * Eq. mu; Sec. 3.2 Listing dmulmod generalised to L words); full-width contexts as stated at
 * moma_ctx_create_full. */
moma_status moma_vec_mulmod(moma_ctx *ctx, size_t n, const uint32_t *a, const uint32_t *b,
                            uint32_t *c, void *stream);

/* out[i] = alpha * x[i] + y[i] mod q (Sec. 2.3, BLAS axpy).  alpha: HOST array of L
 * limbs, canonical.  out may alias y (the BLAS in-place form) or x. */
moma_status moma_vec_axpymod(moma_ctx *ctx, size_t n, const uint32_t *alpha, const uint32_t *x,
                             const uint32_t *y, uint32_t *out, void *stream);

/* ------------------------------------------------------------------ transforms */

/* Forward cyclic NTT of length n (Sec. 2.3 Eq. ntt), natural order in and out:
 * out[k] = sum_j in[j] w_n^(jk) mod q.  n a power of two, 2 <= n <= 2^24, n | q-1,
 * q prime.  in/out: L*n words each; out may equal in. */
moma_status moma_ntt_fwd(moma_ctx *ctx, size_t n, const uint32_t *in, uint32_t *out,
                         void *stream);

/* Inverse: out[j] = n^-1 sum_k in[k] w_n^(-jk) mod q. */
moma_status moma_ntt_inv(moma_ctx *ctx, size_t n, const uint32_t *in, uint32_t *out,
                         void *stream);

/* `count` independent transforms of length n in one launch sequence: transform t reads
 * in + t*L*n and writes out + t*L*n (each transform limb-major on its own).  Launches: one
 * per Stockham pass; a call of little work whose schedule has two passes of at most 8 tiles
 * (128 to 384 bits, count * n up to 2^15 points, 2^16 at 128 bits) runs both passes in one
 * launch of thread-block clusters (one cluster per transform), with no intermediate buffers. */
moma_status moma_ntt_fwd_many(moma_ctx *ctx, size_t n, size_t count, const uint32_t *in,
                              uint32_t *out, void *stream);
moma_status moma_ntt_inv_many(moma_ctx *ctx, size_t n, size_t count, const uint32_t *in,
                              uint32_t *out, void *stream);

/* Cyclic product c = a * b mod (x^n - 1, q) = INTT(NTT(a) . NTT(b)) (Sec. 2.3,
 * polynomial multiplication through the transform); the pointwise product is fused
 * into the first pass of the inverse transform.  a, b, c: L*n words; c may alias a or b. */
moma_status moma_polymul(moma_ctx *ctx, size_t n, const uint32_t *a, const uint32_t *b,
                         uint32_t *c, void *stream);

/* Negacyclic transforms: the ring Z_q[x]/(x^n + 1) of the FHE schemes named in Sec. 1.
 * The paper defines only the cyclic transform (Sec. 2.3 Eq. ntt); this library adds the
 * usual twisted form on top of it.  psi is a primitive 2n-th root of unity with
 * psi^2 = w_n (the root moma_ntt_fwd uses), so 2n must divide q - 1 (else MOMA_ERR_SIZE).
 *   forward: out[k] = sum_j in[j] psi^j w_n^(jk) = in evaluated at psi^(2k+1);
 *   inverse: out[j] = n^-1 psi^-j sum_k in[k] w_n^(-jk), so inverse(forward(x)) = x.
 * The psi^j factor is applied while the first pass loads its input and n^-1 psi^-j while
 * the last pass stores its output (one table of n entries per plan, built on first use).
 * `count` transforms of length n, transform t at in + t*L*n and out + t*L*n, limb-major
 * as everywhere; out may equal in.  count 0 does nothing. */
moma_status moma_ntt_fwd_negacyclic(moma_ctx *ctx, size_t n, size_t count, const uint32_t *in,
                                    uint32_t *out, void *stream);
moma_status moma_ntt_inv_negacyclic(moma_ctx *ctx, size_t n, size_t count, const uint32_t *in,
                                    uint32_t *out, void *stream);

/* Negacyclic product c = a * b mod (x^n + 1, q), through the negacyclic transforms, with
 * the pointwise product fused into the inverse's first pass (as in moma_polymul).
 * a, b, c: L*n words; c may alias a or b.  2n | q - 1. */
moma_status moma_polymul_negacyclic(moma_ctx *ctx, size_t n, const uint32_t *a, const uint32_t *b,
                                    uint32_t *c, void *stream);

/* Same result as moma_ntt_fwd (one transform), but the call allocates no device memory:
 * its intermediate buffers are a fixed 8 MiB array inside the library.  The array is placed
 * on a GPU when the first context on that GPU is created (moma_ctx_create or
 * moma_ctx_create_full, which look up its device address then) and stays there until the
 * process exits.  Meant for callers that may not allocate device memory at call time (memory
 * owned by another allocator under a fixed budget, or a hot path that must not wait on an
 * allocator).  The paper has no counterpart; this is an interface convenience of this
 * library.
 * Limits and conditions:
 *   - L*n <= 2^20 words (n <= 2^19 at 64 bits, 2^18 at 128, 2^17 at 256, 2^16 at 384); larger
 *     n gives MOMA_ERR_SIZE.  Contexts of 512 bits and up give MOMA_ERR_UNSUPPORTED.
 *     Full-width contexts (moma_ctx_create_full) up to 384 bits are accepted.
 *   - The size's twiddle tables must already exist for the forward schedule in effect: call
 *     moma_ntt_fwd once with this context and n beforehand (that call allocates), and again
 *     after any moma_ctx_set_config, moma_autotune or loaded schedule that changes the
 *     forward schedule for this n; otherwise MOMA_ERR_INVALID_ARG.
 *   - The context's device must be current.
 *   - All calls share the one array.  Each call writes every word it later reads, so
 *     nothing needs clearing between calls, but calls that overlap on the GPU (other
 *     streams, other host threads, other contexts) race on it and give wrong results.
 *     out == in is allowed. */
moma_status moma_ntt_fwd_noalloc(moma_ctx *ctx, size_t n, const uint32_t *in, uint32_t *out,
                                 void *stream);

/* ------------------------------------------------------------------ batches */

/* One job of a batch.  op: MOMA_OP_NTT_FWD / NTT_INV (a -> out), MOMA_OP_POLYMUL
 * (out = a * b mod (x^n - 1, q)), MOMA_OP_ADD / SUB / MUL (out = a op b), MOMA_OP_AXPY
 * (out = alpha * a + b, alpha a HOST array of L limbs).  Device vectors follow the
 * conventions above; each job uses its own context (any widths and moduli may be mixed).
 * Jobs at 128 to 384 bits are tiles of the persistent launch; 768-bit jobs and jobs of
 * full-width contexts (moma_ctx_create_full) run with the per-call kernels right after it, on
 * the same stream (and in the same CUDA graph). */
typedef struct {
  int op;
  moma_ctx *ctx;
  size_t n;
  const uint32_t *a;
  const uint32_t *b;
  uint32_t *out;
  const uint32_t *alpha;
} moma_job;

typedef struct moma_batch moma_batch;

/* Prepare a batch (Sec. 5.1: many kernels at once).  Builds the twiddle tables the
 * transforms need, allocates the intermediate buffers, and lays the work out as tiles for
 * one persistent launch: a grid of resident CTAs takes tiles (one pass of one transform,
 * or a slice of one vector op) in dependency order from a device counter; the pointwise
 * product of a cyclic product is fused into the first pass of its inverse.  Job pointers
 * are fixed at creation; refill the same input buffers between runs.  Returns once the
 * batch's descriptors are queued for upload on a library-owned stream (new twiddle tables are
 * built before it returns); every run waits for that upload on its own stream (a stream wait,
 * or a host wait when the caller is capturing the stream into a graph). */
moma_status moma_batch_create(const moma_job *jobs, int njobs, moma_batch **out);

/* Run the batch on `stream` (asynchronous).  The first run launches directly; on a
 * non-default stream the second run captures the launch sequence in a CUDA graph and later
 * runs replay it.  On the legacy default stream, or while the caller is capturing, every run
 * launches directly. */
moma_status moma_batch_run(moma_batch *batch, void *stream);

/* Wait for the device, then return and clear the batch's device-side status:
 * MOMA_ERR_TIMEOUT if a dependency wait ran out (results of the skipped tiles are
 * undefined), else MOMA_OK. */
moma_status moma_batch_sync_status(moma_batch *batch);

/* Bound of every dependency wait, in polls of about 0.1-0.2 us (default 2^24).  A wait
 * that runs out records MOMA_ERR_TIMEOUT and the tile is skipped; the kernel never hangs. */
moma_status moma_batch_set_wait_limit(moma_batch *batch, uint64_t polls);

/* Test hook: make the last queued tile group wait for a completion that never happens,
 * to exercise the bounded wait (the next run reports MOMA_ERR_TIMEOUT). */
moma_status moma_batch_inject_missing_dependency(moma_batch *batch);

/* Release the batch.  Its device memory is returned stream-ordered on an internal stream, so
 * the call does not wait for the device; the caller must make sure no run of the batch is
 * still executing (e.g. synchronise its stream or an event recorded after the last run). */
void moma_batch_destroy(moma_batch *batch);

/* create + run on `stream` + wait + destroy; returns the device-side status. */
moma_status moma_batch_submit(const moma_job *jobs, int njobs, void *stream);

/* ------------------------------------------------------------------ kernel configuration */

/* Operation codes (kernel configuration keys and batch job kinds). */
typedef enum {
  MOMA_OP_NTT_FWD = 0,
  MOMA_OP_NTT_INV = 1,
  MOMA_OP_POLYMUL = 2,
  MOMA_OP_ADD = 3,
  MOMA_OP_SUB = 4,
  MOMA_OP_MUL = 5,
  MOMA_OP_AXPY = 6
} moma_op;

/* Schedule of one operation at one size.  Any field set to 0 means "library default".
 *   engine     1: word products as mad.lo/mad.hi carry chains (mad.lo.cc, madc.hi.cc);
 *              2: word products as mad.wide (whole 64-bit products, carry in the addend);
 *              products by a fixed multiplicand (twiddles, the axpy scalar) form their
 *              truncated high half this way and their low halves by carry chains;
 *              3: (MOMA_OP_MUL only) the double-width product a*b by Karatsuba (Sec. 2.2
 *              Eq. mulk) down to 4-limb carry-chain schoolbook products.
 *              In full-width contexts, MOMA_OP_MUL forms a*b by engine 1, 2 or 3 and reduces it
 *              with a word-based Barrett reduction (an (L+1)-word constant floor(2^(2W)/q));
 *              4: (MOMA_OP_MUL in full-width contexts only) two Montgomery products instead
 *              (REDC(REDC(a b) (R^2 mod q)), Sec. 5.2).  Other ops of full-width contexts
 *              ignore the engine.
 *              1 and 2 compute the same schoolbook sums (Sec. 2.2 Eq. muls, Table 1 mulqdd);
 *              all engines give identical results.
 *   tile_log   transforms: log2 of the elements one CTA holds in shared memory.
 *              BLAS: 0 = operands read with direct vector loads; the width's staged tile
 *              (10 up to 128 bits, 9 at 256 bits, 8 at 384 bits) = operands staged in shared
 *              memory by asynchronous bulk copies (the TMA engine, cp.async.bulk) in tiles of
 *              2^tile_log elements, three tiles in flight per CTA (needs n a multiple of 4 and
 *              16-byte aligned operands, else direct loads); other values are invalid.
 *              Contexts of 512 bits and up and full-width contexts always load directly
 *              (tile_log must be 0 there). 
 *   max_logr   transforms: largest radix (log2) of one Stockham pass.
 *   vec_width  BLAS: elements per thread per step (1, 2 or 4; limited by alignment; full-width
 *              contexts always take 1).
 *   cta_threads transforms: threads per CTA (32, 64, 128 or 256).  Each CTA owns one tile;
 *              small CTAs synchronise fewer warps between butterfly stages.
 *   tight_regs transforms: 1 = kernels compiled for fewer registers per thread (64 up to 256
 *              bits, 102 at 384 bits, 170 at 768 bits) so that more CTAs of at most 128
 *              threads are resident; 0 = no cap beyond the default (85 up to 384 bits).  The
 *              default schedule sets 1 at 384 bits.  Ignored by full-width contexts. */
typedef struct {
  int engine;
  int tile_log;
  int max_logr;
  int vec_width;
  int cta_threads;
  int tight_regs;
} moma_config;

/* Set / read the schedule used for `op` at size n (transforms: exact n; BLAS: every n).
 * moma_ctx_get_config reports the effective schedule (defaults filled in) of one transform
 * per call.  Without a schedule set, a transform call whose count * n is at most 2^19 points
 * (128 to 384 bits) takes a default for little work (2^9-element tiles: 256 threads up to 2^18
 * points, 128 threads with the register cap at 2^19); at 768 bits up to 2^16 points 2^9 tiles
 * and at 2^17 points 2^10 tiles (256 threads); larger calls take the default for large batches.
 * Transforms of a batch (moma_batch_create) that run with the per-call kernels take the schedule
 * of one transform.  Invalid combinations (shared memory over the limit, radix above the tile)
 * give MOMA_ERR_INVALID_ARG. */
moma_status moma_ctx_set_config(moma_ctx *ctx, int op, size_t n, const moma_config *cfg);
moma_status moma_ctx_get_config(moma_ctx *ctx, int op, size_t n, moma_config *cfg);

/* Autotuner: time every candidate schedule of `op` at size n (and `count` transforms for
 * the NTT ops) on scratch buffers of the context's device, with CUDA events on `stream`,
 * keep the fastest in the context (as if set by moma_ctx_set_config) and write it to
 * *best (may be NULL) and its time per call in microseconds to *best_us (may be NULL).
 * Synchronous.  Allocates and frees its scratch buffers; transform plans (twiddle tables) that
 * it builds for candidates other than the winner are freed before it returns. */
moma_status moma_autotune(moma_ctx *ctx, int op, size_t n, size_t count, void *stream,
                          moma_config *best, double *best_us);

/* ------------------------------------------------------------------ word-level blocks */

/* Operations of moma_word_probe. */
typedef enum {
  MOMA_WORD_ADD = 0,     /* out = a + b: L words and the carry word (out plane L)               */
  MOMA_WORD_SUB = 1,     /* out = a - b mod 2^W: L words and the borrow (out plane L)            */
  MOMA_WORD_MUL = 2,     /* out = a * b: 2L words (engine 1 carry chains, 2 whole products,
                            3 Karatsuba)                                                         */
  MOMA_WORD_MUL_HI = 3,  /* out = the truncated high half floor(a*b / 2^W) or one less: L words
                            (engine 1 or 2)                                                      */
  MOMA_WORD_BARRETT = 4, /* out = a * b mod q by Barrett reduction (L words), plane L = 1 when the
                            final correction fired (Barrett contexts; a, b canonical)            */
  MOMA_WORD_FIXED = 5,   /* out = a * w - s * q with w = b's element 0 and s the quotient estimate
                            from w's companion, before any correction: in [0, 3q) (Barrett
                            contexts; w canonical; a any L-word value; engine 1 or 2 as for
                            the transforms' twiddle products)                                    */
  MOMA_WORD_MONT = 6,    /* out = a * b * R^-1 mod q, R = 2^W (full-width contexts; a, b < q)     */
  MOMA_WORD_BARRETT_FULL = 7 /* planes 0..L: r = a*b - s*q before the final subtractions, L+1 words,
                            in [0, 4q) (s the truncated quotient estimate from floor(2^(2W)/q));
                            planes L+1..2L: a * b mod q.  Full-width contexts; a, b < q; the
                            product a*b by `engine` (1, 2 or 3)                                  */
} moma_word_op;

/* The word-level building blocks of the multi-word arithmetic (Sec. 3, Table 1 rules;
 * Sec. 2.2 Eq. muls / Eq. mulk; Sec. 3.1 Eq. barrett), one element per thread, with their raw
 * outputs, for tests that check each block against integer arithmetic and against the bounds
 * the method relies on.  a, b: L*n words (limb-major, device); out: (2L+1)*n words
 * (limb-major, device; planes not written by the operation are zero).  The context supplies
 * the modulus and its constants; MOMA_WORD_BARRETT and MOMA_WORD_FIXED need a context made by
 * moma_ctx_create, MOMA_WORD_MONT and MOMA_WORD_BARRETT_FULL one made by moma_ctx_create_full (else
 * MOMA_ERR_INVALID_ARG).  64 to 768 bits (1024-bit contexts give MOMA_ERR_UNSUPPORTED).
 * n <= 2^30.  Asynchronous on `stream`, except MOMA_WORD_FIXED, which first reads w from the
 * device. */
moma_status moma_word_probe(moma_ctx *ctx, int op, int engine, size_t n, const uint32_t *a,
                            const uint32_t *b, uint32_t *out, void *stream);

/* ------------------------------------------------------------------ measurement */

/* Integer multiply-add issue-rate microbenchmark (used for the compute roofline).
 * Runs `blocks` x `threads` threads (threads <= 256), each issuing `iters` rounds of 64
 * multiply instructions of one PTX form: 0 carry-chain rows (mad.lo.cc/madc.lo.cc then
 * mad.hi.cc/madc.hi.cc, 8 independent chains), 1 the same as one dependent chain,
 * 2 mad.lo/mad.hi alternating, 3 mad.lo only, 4 mad.hi only, 5 mad.wide.u32, 6 lo
 * carry rows only, 7 hi carry rows only, 8 add.cc chains (no multiply), 9 rows as plain
 * 64-bit C arithmetic (64 word products).  Writes the kernel time in milliseconds and
 * 64 * iters * blocks * threads (the operations issued at the PTX/C level).
 * Synchronous (uses the legacy default stream). */
moma_status moma_probe_imad(int variant, int blocks, int threads, int iters, double *ms_out,
                            double *imad_out);

#ifdef __cplusplus
}
#endif

#endif /* MOMA_H */
