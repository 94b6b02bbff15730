/*
 * velopir.h -- C ABI of libvelopir.so: batched TFHE gate bootstrapping on one
 * GB300 (sm_103a) and the server-side circuits of VeLoPIR's three query modes.
 * Key generation, encryption, decryption and Alg. PubKeyGen / ServerEnc are
 * in the separate host-only library libvelopir_client.so (velopir_client.h),
 * which needs no GPU and no CUDA runtime; the same computations also run here
 * as CUDA kernels (velopir_gpu_*), bit-identical, for a key that should stay
 * on the device and for Alg. ServerEnc over a large database.
 *
 * Paper: "Versatile and Fast Location-Based PIR with FHE over the Torus"
 * (VeLoPIR).  Section 2.2 defines TLWE encryption, Ecd, Dec and the gate
 * HomAND = Bootstrap((0,-1/8) + ct1 + ct2); Bootstrap = BlindRotate,
 * SampleExtract, KeySwitch with internals from tfhe-2 (Chillotti et al.,
 * J. Cryptol. 2020); parameters from the Appendix table (n = 630, N = 1024,
 * k = 1, l = 3, Bg = 2^7, key-switch base 2^2 with t = 8 levels).
 *
 * Conventions shared by every entry point:
 *  - Torus values are uint32_t with 1.0 == 2^32; all arithmetic is mod 2^32.
 *  - An LWE ciphertext is 631 contiguous uint32_t: a[0..629] then b.
 *  - A multi-bit value is an array of bit ciphertexts, least significant bit
 *    first (ct[i] encrypts bit i).
 *  - Every function returns 0 (VELOPIR_OK) or a negative VELOPIR_ERR_* code;
 *    velopir_last_error() then describes the failure.  No function aborts.
 *  - Buffers belong to the caller.  A pointer may be host or device memory
 *    (classified with cudaPointerGetAttributes); results are written to the
 *    memory kind the caller passed.  Host ciphertext buffers are staged
 *    through device scratch owned by the context; plaintext databases are
 *    read on the host (the scheduler compiles them into the gate program),
 *    so a device-resident database is first copied to the host.
 *  - Calls on one context are serialised on the context's CUDA stream and are
 *    synchronous unless stated otherwise (velopir_submit is asynchronous).
 *  - A context is not thread-safe; use one context per host thread.  The
 *    exception is serving with the issue thread (velopir_serve_start): the
 *    serving calls may then come from any thread.
 */
#ifndef VELOPIR_H
#define VELOPIR_H

#include <stddef.h>
#include <stdint.h>

#include "velopir_common.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Gates (Section 2.2 names HomAND, HomXOR, HomXNOR; the others are tfhe-2's
 * gate set under the same encoding).  Each binary gate is one bootstrap of a
 * linear pre-combination; MUX(c, a, b) = c ? a : b uses two blind rotations
 * and one key switch. */
typedef enum {
    VP_AND = 0, VP_NAND, VP_OR, VP_NOR, VP_XOR, VP_XNOR,
    VP_ANDNY, /* (NOT c1) AND c2 */
    VP_ANDYN, /* c1 AND (NOT c2) */
    VP_ORNY,  /* (NOT c1) OR c2  */
    VP_ORYN,  /* c1 OR (NOT c2)  */
    VP_MUX
} velopir_gate;

/* Implementation of the external product inside blind rotation.  Every path
 * returns bit-identical ciphertexts; they differ only in speed. */
typedef enum {
    VP_PATH_INT32_DENSE = 0, /* dense negacyclic contraction on the integer pipe */
    VP_PATH_NTT = 1,         /* exact two-prime number-theoretic transform (default) */
    VP_PATH_TENSOR_F16 = 2   /* exact small-integer limbs on tcgen05 kind::f16 */
} velopir_path;

typedef struct velopir_ctx velopir_ctx;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may allocate (keys + scratch); 0 = no cap.  cuda_stream
 * (a cudaStream_t, nullable) is the stream every launch goes to; NULL makes
 * the context create and own a non-blocking stream.  *out is set to NULL on
 * failure.  Errors: ERR_ARG, ERR_NOCUDA, ERR_CUDA. */
int velopir_create(velopir_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream);

/* Release every device allocation of the context and the context itself.
 * Waits for outstanding work first.  NULL is accepted. */
int velopir_destroy(velopir_ctx *ctx);

/* Upload the cloud key (Section 2.2 KeyGen's evaluation key evk).
 *   bk : bootstrapping key, uint32_t[630][6][2][1024]; entry [i][r][j] is
 *        component j (0 = a(X), 1 = b(X)) of TRGSW row r = 2(p-1)+q of
 *        BK_i = TRGSW_K(s_i) (level p = 1..3, component q), coefficients
 *        in increasing degree.  bk_words must be 630*6*2*1024.
 *   ksk: key-switching key, uint32_t[1024][8][4][631]; entry [i][j][v] is
 *        LWE_s(v * K_i * 2^(32-2(j+1))).  ksk_words must be 1024*8*4*631.
 * The library keeps device copies in its own layout (padded KSK rows, the
 * transformed BK of the selected path).  Replaces a previously loaded key.
 * Errors: ERR_ARG (params not the paper's set, wrong sizes), ERR_OOM, ERR_CUDA. */
int velopir_load_cloud_key(velopir_ctx *ctx, const velopir_params *params,
                           const uint32_t *bk, size_t bk_words,
                           const uint32_t *ksk, size_t ksk_words);

/* Select the external-product implementation (default VP_PATH_NTT).  The key
 * stays loaded: the path's transformed copy of BK is built on the device the
 * first time the path runs.  Errors: ERR_ARG (unknown or unavailable path). */
int velopir_set_path(velopir_ctx *ctx, velopir_path path);

/* Cap the blind rotations per kernel launch (default and maximum 65,536; 0
 * restores the default).  A layer larger than the cap runs as several
 * launches; a MUX's two rotations always share one.  max_rotations = 1 is the
 * plain one-bootstrap-per-launch execution of any query or batch, the
 * baseline that layer batching is measured against.  Results are identical
 * under every cap.  Errors: ERR_ARG. */
int velopir_set_launch_limit(velopir_ctx *ctx, size_t max_rotations);

/* Fan-in of the XOR aggregation tree of the *_encdb calls with a payload
 * (default 2; 0 restores it).  2 is Section 5's pairwise HomSum, (D-1) l_S
 * bootstraps; g in 3..8 XORs g values with one bootstrap
 * of 2 sum c_k + T((g-1)/4), ceil((D-1)/(g-1)) l_S bootstraps at most, in
 * ceil(log_g D) levels.  The plaintext answer is the same for every g; the
 * noise margin falls with g (about 18 sigma at 2, 9 sigma at 8).
 * Errors: ERR_ARG, ERR_BUSY. */
int velopir_set_encdb_fanin(velopir_ctx *ctx, int fanin);

/* One gate on each of `count` independent inputs, all bootstraps issued as
 * one batch (blind rotation of every input shares each step's BK_i).
 *   lwe_in : uint32_t[count][arity][631], arity 2 (3 for VP_MUX: c, a, b)
 *   lwe_out: uint32_t[count][631]
 * count == 0 is a no-op.  Errors: ERR_ARG, ERR_NOKEY, ERR_OOM, ERR_CUDA,
 * ERR_TIMEOUT. */
int velopir_bootstrap_batch(velopir_ctx *ctx, velopir_gate gate, const uint32_t *lwe_in,
                            uint32_t *lwe_out, size_t count);

/* Largest batch velopir_bootstrap_batch_noalloc accepts. */
#define VELOPIR_NOALLOC_MAX_GATES 256

/* velopir_bootstrap_batch for callers that cannot allocate device memory at
 * call time: a serving process that reserved its HBM at start-up, code under
 * a hard memory cap or behind a caching allocator that must not see foreign
 * allocations, or a latency-critical loop where cudaMalloc/cudaFree (cudaFree
 * synchronises the device) would stall other work.  The paper has no
 * counterpart; this is a deployment variant of the same computation and
 * returns bit-identical ciphertexts.
 *
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * Its scratch (job lists and extracted rows, 2.1 MB) is one file-scope device
 * array of the library that every device loading the library holds until the
 * process exits.  All calls share that array; calls whose GPU work overlaps
 * race, so serialise them (one stream, or events).  Nothing in it needs
 * clearing: each call writes every word it reads.
 *   lwe_in, lwe_out: device memory, layouts as velopir_bootstrap_batch.
 *   count: 0 .. VELOPIR_NOALLOC_MAX_GATES; larger counts return ERR_ARG.
 * The context's key must be loaded (keys are allocated at load time, not
 * here).  The selected path is used once its transformed key exists (after
 * the context's first bootstrap or query on that path); before that the dense
 * path runs; all paths give the same bits.
 * The first call on a device performs a one-time set-up (it looks up the
 * array's device address with that device current), so make that first call
 * before any CUDA stream capture.  Synchronous: returns after the stream has
 * finished the work.  Its status includes the context's device error word,
 * as every synchronous call's does: a bounded wait that gave up in earlier
 * asynchronous work on the same context (serving steps) is reported by the
 * next synchronous call, which may be this one.  Errors: ERR_ARG (sizes,
 * null or host pointers, unknown gate), ERR_NOKEY, ERR_CUDA, ERR_TIMEOUT. */
int velopir_bootstrap_batch_noalloc(velopir_ctx *ctx, velopir_gate gate, const uint32_t *lwe_in,
                                    uint32_t *lwe_out, size_t count);

/* The same gates issued one bootstrap per kernel launch (no batching): the
 * "plain" baseline against which batching is measured.  Same arguments. */
int velopir_bootstrap_plain(velopir_ctx *ctx, velopir_gate gate, const uint32_t *lwe_in,
                            uint32_t *lwe_out, size_t count);

/* IntV (Alg. InterValid) against a plaintext database of D rectangles.
 *   enc_x, enc_y: uint32_t[32][631] each, bitwise encryptions of unsigned
 *                 32-bit coordinates x and y.
 *   rects       : uint32_t[D][4] = x_lo, x_hi, y_lo, y_hi (plaintext, unsigned)
 *   out_bits    : uint32_t[D][631]; entry d encrypts
 *                 x_lo <= x < x_hi AND y_lo <= y < y_hi (half-open, Theorem bb1).
 * Comparators follow Alg. HomCompLeOPT with XNOR/MUX against plaintext bits
 * rewritten into single gates and the top bit flipped for unsigned order;
 * 131 bootstraps per entry in 34 gate layers; the list scheduler launches
 * the ready gates of all entries as whole waves of the blind-rotation kernel.
 * Errors: ERR_ARG, ERR_NOKEY, ERR_OOM, ERR_CUDA, ERR_TIMEOUT. */
int velopir_interval_query(velopir_ctx *ctx, const uint32_t *enc_x, const uint32_t *enc_y,
                           const uint32_t *rects, size_t D, uint32_t *out_bits);

/* CoV (Alg. CoV with Alg. HomEqOPT) against D plaintext grid cells.
 *   enc_cell: uint32_t[32][631]: bits 0..15 encrypt x, bits 16..31 encrypt y.
 *   cells   : uint32_t[D], packed (y << 16) | x.
 *   out_bits: uint32_t[D][631]; entry d encrypts (x, y) == cell d.
 * 31 bootstraps per entry in 5 gate layers.  Errors as above. */
int velopir_coordinate_query(velopir_ctx *ctx, const uint32_t *enc_cell, const uint32_t *cells,
                             size_t D, uint32_t *out_bits);

/* IdM: Alg. HomEqOPT of an encrypted identifier against D plaintext ids.
 *   enc_id : uint32_t[id_bits][631], 1 <= id_bits <= 32.
 *   ids    : uint32_t[D] (only the low id_bits bits are compared).
 *   payload: NULL, or uint32_t[D] plaintext payloads.
 *   out    : payload == NULL: uint32_t[D][631] match bits.
 *            payload != NULL: uint32_t[payload_bits][631], the HomSum of the
 *            zeroed-out payloads (Alg. HomBitwiseAND with a plaintext
 *            payload, then the pairwise XOR reduction of Section 5), i.e. an
 *            encryption of the payload of the matching entry (0 if none).
 *   1 <= payload_bits <= 32.  Errors as above. */
int velopir_id_match(velopir_ctx *ctx, const uint32_t *enc_id, int id_bits, const uint32_t *ids,
                     size_t D, const uint32_t *payload, int payload_bits, uint32_t *out);

/* ---- encrypted database (the paper's protocol) ----------------------------- */

/* Section 3.2's preprocessing encrypts the database under the client's key:
 * Alg. PubKeyGen gives the server one fresh encryption of zero per database
 * bit, Alg. ServerEnc adds the encoded bit to it.  The query then runs
 * Section 4-5's circuits with both operands encrypted: equality tests
 * bootstrap their XNORs, comparators their XNORs and MUXes (Alg. HomCompLeOPT:
 * t0 = XOR of the top bits, t1 = MUX(XNOR(c1_i, c2_i), t1, c2_i) for
 * i = 0..l-2, result MUX(t0, c1_top, t1); two blind rotations per MUX), and
 * an encrypted payload is zeroed with a bootstrapped AND (Alg.
 * HomBitwiseAND).  Ciphertext arrays may be host or device memory; outputs
 * as in the plaintext-database calls. */

/* The database ciphertexts come from Alg. PubKeyGen and Alg. ServerEnc,
 * which run on the host (velopir_client.h). */

/* Largest encrypted payload (bits per entry) of the encdb calls. */
#define VELOPIR_MAX_ENC_PAYLOAD_BITS 4096

/* Every encdb call has the same payload convention.  enc_payload == NULL:
 * out = [D][631], one validation bit per entry.  Otherwise enc_payload =
 * [D][payload_bits][631] (1 <= payload_bits <= VELOPIR_MAX_ENC_PAYLOAD_BITS,
 * the paper's l_S), each entry's payload is zeroed by its validation bit with
 * one bootstrapped AND per bit (Alg. HomBitwiseAND) and the D results are
 * XOR-aggregated by a tree of the context's fan-in (velopir_set_encdb_fanin;
 * by default pairwise, Section 5's HomSum, (D-1) payload_bits bootstraps):
 * out = [payload_bits][631], the XOR of the payloads of the valid entries. */

/* IntV over an encrypted database (Alg. InterValid): validation bit
 * (x_lo <= x < x_hi && y_lo <= y < y_hi) for l-bit unsigned coordinates
 * (1 <= l <= 32; the paper's interval precision l_I).  enc_x, enc_y:
 * [l][631]; enc_rects: [D][4][l][631] (x_lo, x_hi, y_lo, y_hi, bits LSB
 * first).  12 l + 3 bootstraps per entry (per comparator: 1 XOR, l-1 XNORs,
 * l MUXes of 2).  Errors: ERR_ARG, ERR_NOKEY, ERR_OOM, ERR_CUDA, ERR_TIMEOUT. */
int velopir_interval_query_encdb(velopir_ctx *ctx, const uint32_t *enc_x, const uint32_t *enc_y, int l,
                                 const uint32_t *enc_rects, size_t D, const uint32_t *enc_payload,
                                 int payload_bits, uint32_t *out);

/* CoV over an encrypted database (Alg. CoV with Alg. HomEqOPT): validation
 * bit (cell == cell_d).  enc_cell: [2w][631] (w bits of x, then w bits of y;
 * 1 <= w <= 16), enc_cells: [D][2w][631].  4 w - 1 bootstraps per entry.
 * Errors: as above. */
int velopir_coordinate_query_encdb(velopir_ctx *ctx, const uint32_t *enc_cell, int w, const uint32_t *enc_cells,
                                   size_t D, const uint32_t *enc_payload, int payload_bits, uint32_t *out);

/* IdM over an encrypted database: validation bit (id == id_d).  enc_id:
 * [id_bits][631] (1..32 bits), enc_ids: [D][id_bits][631].  2 id_bits - 1
 * bootstraps per entry.  Errors: as above. */
int velopir_id_match_encdb(velopir_ctx *ctx, const uint32_t *enc_id, int id_bits, const uint32_t *enc_ids,
                           size_t D, const uint32_t *enc_payload, int payload_bits, uint32_t *out);

/* ---- several queries as one program --------------------------------------- */

typedef enum { VP_QUERY_INTV = 0, VP_QUERY_COV = 1, VP_QUERY_IDM = 2 } velopir_query_kind;

typedef struct {
    int32_t kind;            /* velopir_query_kind */
    int32_t id_bits;         /* IdM only */
    int32_t payload_bits;    /* IdM with payload only */
    int32_t agg_fanin;       /* IdM with payload: fan-in of the XOR aggregation tree.  0 or 2 is
                                Section 5's pairwise HomSum (D - 1 bootstraps per payload bit);
                                g in 3..8 XORs g values with one bootstrap of
                                2 (c_1 + ... + c_g) + T((g-1)/4), whose phase is +-1/4 by the
                                parity of the true inputs (about (D - 1)/(g - 1) bootstraps per
                                bit).  The doubled input noise against the 1/4 margin stays
                                above 9 standard deviations of tfhe-2's output-noise bound up to
                                g = 8.  Same plaintext result, different ciphertexts.
                                velopir_plan_query also takes it for the VP_PLAN_*_ENCDB kinds
                                (the fan-in velopir_set_encdb_fanin sets). */
    const uint32_t *enc_a;   /* IntV: enc_x; CoV: enc_cell; IdM: enc_id (host or device) */
    const uint32_t *enc_b;   /* IntV: enc_y; otherwise NULL */
    const uint32_t *db;      /* rects / cells / ids (host or device; copied at submit) */
    const uint32_t *payload; /* IdM payloads (host or device; copied at submit) or NULL */
    size_t D;
    uint32_t *out;           /* result buffer, same shapes as the synchronous calls */
} velopir_query;

/* Run nq queries (of any modes and database sizes) as one gate program: the
 * layers of all queries are packed into shared launches (Section 5's
 * outermost parallelism across entries, extended across queries).  Buffers
 * as in velopir_submit; results are in each q->out on return.  use_graph != 0
 * captures the launch sequence into a CUDA graph and replays it while the
 * next batch has the same launch list (same modes, sizes and plaintext
 * shapes).  Errors: as the synchronous query calls. */
int velopir_query_batch(velopir_ctx *ctx, const velopir_query *queries, size_t nq, int use_graph);

/* How many times a captured graph was replayed instead of re-captured. */
uint64_t velopir_graph_replays(velopir_ctx *ctx);

/* Autotuner of the blind-rotation tile shape (bootstraps per CTA: 6, 8, 9,
 * 10 or 12 for the NTT path).  Times one full wave of each shape on the device and keeps
 * the results for this process; afterwards every launch of `count`
 * bootstraps uses the shape with the fewest (waves x measured wave time), so
 * uneven layer sizes waste fewer SMs.  wave_ms_out (nullable, n_out entries)
 * receives the measured wave times in ms, smallest shape first.  A no-op on the
 * dense path.  Errors: ERR_NOKEY, ERR_OOM, ERR_CUDA, ERR_TIMEOUT. */
int velopir_autotune(velopir_ctx *ctx, double *wave_ms_out, int n_out);

/* Bootstraps per CTA the current path would use for a batch of `count`
 * (>= 1 on success).  Errors: ERR_ARG. */
int velopir_tuned_shape(velopir_ctx *ctx, size_t count);

/* Kinds accepted by velopir_plan_query only: the three modes over an
 * encrypted database (the *_encdb calls).  q->id_bits is then the width
 * (IntV l, CoV w, IdM id_bits), db and payload hold plaintext values (IntV
 * [D][4], CoV [D] packed (y << w) | x, IdM [D]; payload [D], payload_bits
 * <= 32), and the dry run encrypts every database bit as a ServerEnc
 * ciphertext would be. */
#define VP_PLAN_INTV_ENCDB 3
#define VP_PLAN_COV_ENCDB 4
#define VP_PLAN_IDM_ENCDB 5

/* Host-only dry run of a query's launch plan; no GPU or context is used.
 * Builds the gate program of q (Section 5's circuits for IntV, CoV or IdM,
 * with q->kind, D, db, id_bits, payload and payload_bits as in the query
 * calls; enc_a, enc_b and out are ignored), schedules it as the device path
 * does -- launches of whole waves of `wave` blind rotations when at least a
 * wave is ready, longest dependency chain first (wave = 0: one launch per
 * as-soon-as-possible layer) -- assigns pool slots, and executes it on
 * noiseless plaintext phases instead of ciphertexts: each ciphertext is its
 * message +-1/8 (Section 2.2 Ecd) and each bootstrap returns the message of
 * the sign of its pre-combined phase (phase 0 reads as true).
 *   bits_a: the query's plaintext bits, one uint32_t 0/1 per ciphertext of
 *           enc_a (IntV x[32] or x[l], CoV cell[32] or cell[2w], IdM
 *           id[id_bits]), LSB first;
 *   bits_b: IntV y[32] or y[l], else ignored (nullable);
 *   bits_out: receives one 0/1 per output ciphertext (D entries, or
 *             payload_bits with a payload);
 *   launch_sizes (nullable): receives the blind rotations of each launch
 *           (one entry per scheduled layer, before the executor splits a
 *           layer into chunks), up to max_launches entries.
 * Returns the number of launches (>= 1), VELOPIR_ERR_ARG for bad arguments,
 * or VELOPIR_ERR_PLAN if any gate of the plan would read a value that is not
 * yet written or whose pool slot was already reused. */
int velopir_plan_query(const velopir_query *q, int wave, const uint32_t *bits_a, const uint32_t *bits_b,
                       uint32_t *bits_out, size_t *launch_sizes, int max_launches);

/* Host-only dry run of a batch of queries as velopir_query_batch runs them:
 * one merged gate program over all queries, scheduled as in
 * velopir_plan_query, executed in the device's launch order -- each launch
 * split into chunks of at most chunk_rows blind rotations (0: no split;
 * the executor splits at 65,536; like the executor, the dry run never uses
 * fewer than 2 rows, so a MUX's two rotations share a chunk), a layer's
 * multi-input sums first and every chunk's blind rotations before its key
 * switches -- on noiseless plaintext phases.  launch_sizes holds the blind
 * rotations per scheduled layer, as in velopir_plan_query.  Plaintext-database kinds
 * (VP_QUERY_*) only.  bits_a, bits_b and bits_out are the per-query arrays
 * of velopir_plan_query concatenated in query order (bits_b holds the IntV
 * queries' y bits only).  Returns the number of launches, ERR_ARG, or
 * ERR_PLAN as velopir_plan_query. */
int velopir_plan_batch(const velopir_query *qs, size_t nq, int wave, int chunk_rows, const uint32_t *bits_a,
                       const uint32_t *bits_b, uint32_t *bits_out, size_t *launch_sizes, int max_launches);

/* ---- serving: asynchronous queries with continuous batching ------------- */

/* Enqueue a query.  It is admitted into the running batch as soon as the
 * context's HBM budget allows; its gate layers are merged with those of every
 * other admitted query into shared launches.  *ticket identifies it.  The
 * caller must not touch enc_*, db, payload or out until velopir_poll reports
 * done.  Errors: ERR_ARG, ERR_NOKEY, ERR_BUSY (queue full). */
int velopir_submit(velopir_ctx *ctx, const velopir_query *q, uint64_t *ticket);

/* Advance the serving loop by at most one merged layer launch and report
 * whether `ticket` has finished (*done = 1; its result is in q->out).
 * Errors: ERR_ARG (unknown ticket), ERR_CUDA, ERR_TIMEOUT. */
int velopir_poll(velopir_ctx *ctx, uint64_t ticket, int *done);

/* Cancel a submitted query.  A waiting query is dropped at once; an admitted
 * one gets no further launches, and its memory is released when the work
 * already issued for it has finished.  The ticket is then reported like a
 * finished one, and velopir_poll returns VELOPIR_ERR_CANCELLED for it (with
 * *done = 1); its output is undefined.  Until then the query's buffers may
 * still be read or written by work already on the device.  A query whose last
 * layer is already issued completes normally.  Errors: ERR_ARG (unknown
 * ticket), ERR_CUDA. */
int velopir_cancel(velopir_ctx *ctx, uint64_t ticket);

/* Advance the serving loop by at most one merged layer launch (admitting
 * waiting queries first) and report up to `cap` tickets that have finished
 * since the last report (*ndone of them, written to done[]).  A ticket
 * reported here is not reported again by velopir_poll.  Errors: ERR_ARG,
 * ERR_CUDA, ERR_TIMEOUT. */
int velopir_progress(velopir_ctx *ctx, uint64_t *done, size_t cap, size_t *ndone);

/* Start the context's issue thread, a host thread owned by the library that
 * admits waiting queries and issues serving steps back to back, keeping up
 * to two steps queued on the stream, so the GPU never waits for the caller
 * between steps.  While it runs: velopir_submit, velopir_cancel,
 * velopir_queue_depth, velopir_poll and velopir_progress may be called from
 * any host thread (poll and progress then only report: they issue nothing);
 * every other call on this context returns ERR_BUSY.  A failure of the
 * thread (ERR_TIMEOUT from a serving step, ERR_CUDA) is returned by the next
 * poll or progress.  Errors: ERR_ARG, ERR_NOKEY, ERR_OOM, ERR_CUDA. */
int velopir_serve_start(velopir_ctx *ctx);

/* Stop the issue thread once the steps already issued have finished.
 * Queries still waiting or admitted stay; velopir_poll and
 * velopir_progress step them again.  Returns the thread's first failure, if
 * any.  velopir_destroy stops the thread first.  Errors: ERR_ARG,
 * ERR_TIMEOUT, ERR_CUDA. */
int velopir_serve_stop(velopir_ctx *ctx);

/* Number of admitted and waiting queries.  Errors: ERR_ARG. */
int velopir_queue_depth(velopir_ctx *ctx, size_t *admitted, size_t *waiting);

/* Wait for all work on the context's stream.  Errors: ERR_CUDA, ERR_TIMEOUT. */
int velopir_sync(velopir_ctx *ctx);

/* Message of the last failure on this context ("" if none), as a copy owned
 * by the calling thread that stays valid until that thread's next call of
 * this function (the issue thread may record a failure meanwhile).  NULL ctx
 * gives the last failure of velopir_create on this thread. */
const char *velopir_last_error(velopir_ctx *ctx);

/* Kernel launches this context has issued since creation (for launch counting). */
uint64_t velopir_launch_count(velopir_ctx *ctx);

/* Failure-detection self-test: launches the library's bounded device wait on
 * a barrier nothing ever completes.  The wait gives up after its time limit
 * (2 s), the kernel returns normally, and the call returns
 * VELOPIR_ERR_TIMEOUT; the context stays usable (the error word is cleared).
 * Returns VELOPIR_OK only if the wait did not time out, which is a defect. */
int velopir_selftest_wait_timeout(velopir_ctx *ctx);

/* ---- tracing: per-kernel device time -------------------------------------- */

typedef enum {
    VP_KERNEL_BLIND_ROTATE = 0,
    VP_KERNEL_KEY_SWITCH = 1,
    VP_KERNEL_FREE = 2,    /* bootstrap-free gates */
    VP_KERNEL_SUM = 3,     /* multi-input pre-combinations of the fan-in aggregation */
    VP_KERNEL_TRACE = 4    /* gate-trace copies (velopir_trace_start) */
} velopir_kernel;

/* enable != 0: bracket every subsequent kernel launch with CUDA events on the
 * context's stream and accumulate its device time per kernel kind; 0 stops.
 * Enabling also clears the accumulated totals.  Errors: ERR_ARG, ERR_CUDA. */
int velopir_profile(velopir_ctx *ctx, int enable);

/* Totals since profiling was enabled for one kernel kind: launches, work
 * units (bootstraps for blind rotation, gates for key switch, ciphertexts
 * for free gates) and device milliseconds.  Synchronises the stream.
 * Errors: ERR_ARG, ERR_CUDA. */
int velopir_profile_read(velopir_ctx *ctx, int kernel, uint64_t *launches, uint64_t *units, double *ms);

/* ---- gate trace: per-gate records for parity checks ---------------------- */

#define VELOPIR_TRACE_MAX_IN 8

/* One executed gate as the device ran it.  The gate is Bootstrap of linear
 * pre-combinations (Section 2.2's gate form; MUX per tfhe-2): rotation
 * r < nrot blind-rotates c_r = sum_{k < nin} coef[r][k] * in[k] + T(cst[r])
 * and extracts it; the extractions are summed, T(ks_cst) is added, and the
 * sum is key-switched into out.  Bootstrap-free gates folded into a gate's
 * inputs show up as its coefficients and constants; a multi-input sum of the
 * fan-in aggregation is expanded into its terms.  in[k] for k >= nin is
 * zero.  22,800 bytes. */
typedef struct {
    uint32_t nrot;                                       /* 1, or 2 for MUX */
    uint32_t nin;                                        /* distinct inputs, <= 8 */
    uint32_t ks_cst;                                     /* torus constant before key switching */
    uint32_t cst[2];                                     /* torus constant of each rotation */
    int32_t coef[2][VELOPIR_TRACE_MAX_IN];               /* coefficient of in[k] in rotation r */
    uint32_t in[VELOPIR_TRACE_MAX_IN][VELOPIR_LWE_WORDS];/* inputs as the gate read them */
    uint32_t out[VELOPIR_LWE_WORDS];                     /* the gate's output */
} velopir_trace_rec;

/* ---- Client-side preprocessing on the GPU -------------------------------
 * The computations of libvelopir_client.so (velopir_client.h) run as CUDA
 * kernels, from the same caller-supplied random numbers, with bit-identical
 * results: a cloud key generated here can be passed (device pointers) straight
 * to velopir_load_cloud_key, and a server can run Alg. ServerEnc over a large
 * database on the device that evaluates it.  Every buffer may be host or
 * device memory; host buffers are staged through stream-ordered temporaries
 * (cudaMallocAsync) released before the call returns and not counted against
 * the context's HBM budget -- pass device buffers to avoid them.  The
 * context's key need not be loaded.
 * Synchronous.  Errors: ERR_ARG (null buffer, other parameters, count above
 * 2^24), ERR_OOM (staging), ERR_CUDA, ERR_BUSY (the issue thread runs). */

/* Section 2.2 KeyGen of the cloud key: BK_i row r = 2(p-1)+q is the TRLWE
 * sample (a, a K + e) under the TRLWE key K, plus s_i 2^(32-7p) on component q
 * (TRGSW encryption of s_i, Bg = 2^7); KSK[i][j][v] = (a, <a, s> + v K_i
 * 2^(32-2(j+1)) + e).  Inputs and outputs as velopir_client_keygen:
 * s[630], K[1024] key bits (0/1), bk_a/bk_e uint32_t[630][6][1024],
 * ksk_a uint32_t[1024][8][4][630], ksk_e uint32_t[1024][8][4]; bk_out
 * uint32_t[630][6][2][1024], ksk_out uint32_t[1024][8][4][631]. */
int velopir_gpu_keygen(velopir_ctx *ctx, const velopir_params *params, const uint32_t *s, const uint32_t *K,
                       const uint32_t *bk_a, const uint32_t *bk_e, const uint32_t *ksk_a, const uint32_t *ksk_e,
                       uint32_t *bk_out, uint32_t *ksk_out);

/* Section 2.2 Enc with Ecd (1 -> 1/8, 0 -> -1/8): out_c = (a_c, <a_c, s> +
 * Ecd(bits_c) + e_c).  s uint32_t[630] (0/1), bits uint32_t[count], a
 * uint32_t[count][630], e uint32_t[count], out uint32_t[count][631].
 * count == 0 is a no-op. */
int velopir_gpu_encrypt_bits(velopir_ctx *ctx, const uint32_t *s, const uint32_t *bits, const uint32_t *a,
                             const uint32_t *e, size_t count, uint32_t *out);

/* Alg. PubKeyGen: count encryptions of zero, pk_c = (a_c, <a_c, s> + e_c);
 * layouts as velopir_gpu_encrypt_bits. */
int velopir_gpu_pubkeygen(velopir_ctx *ctx, const uint32_t *s, const uint32_t *a, const uint32_t *e, size_t count,
                          uint32_t *pk_out);

/* Alg. ServerEnc: ct_c = (0, Ecd(bits_c)) + pk_c.  pk and ct_out
 * uint32_t[count][631], bits uint32_t[count] (0/1).  Uses no secret. */
int velopir_gpu_server_encrypt(velopir_ctx *ctx, const uint32_t *pk, const uint32_t *bits, size_t count,
                               uint32_t *ct_out);

/* Start recording a sample of the gates that this context's programs and
 * serving steps execute (velopir_bootstrap_batch, the query calls,
 * velopir_query_batch with or without graph capture, velopir_submit; not
 * velopir_bootstrap_batch_noalloc).  Of every launch of G blind-rotated
 * gates, max(min(per_launch, G), ceil(G / one_in)) gates (one_in = 0: only
 * the per-launch count), chosen uniformly by a generator seeded with `seed`,
 * are copied into a device buffer of `cap` records (reserved here, counted
 * against the HBM budget) right after their key switch; once `cap` records
 * are written, further gates are not recorded.  The per-launch count reaches
 * every level of every circuit, including the few-gate top levels of an
 * aggregation tree; one_in spreads the rest over the large launches.
 * Restarting discards the previous records.  Errors: ERR_ARG (per_launch =
 * one_in = 0, cap = 0 or cap > 2^20), ERR_OOM, ERR_CUDA. */
int velopir_trace_start(velopir_ctx *ctx, uint64_t seed, uint32_t per_launch, uint32_t one_in, size_t cap);

/* Stop recording; copy the first min(cap, recorded) records to out (host or
 * device memory, nullable when cap = 0), set *count to the number recorded,
 * and release the buffer.  Synchronises the stream.  Errors: ERR_ARG,
 * ERR_CUDA, ERR_TIMEOUT (a device wait of a traced program gave up). */
int velopir_trace_stop(velopir_ctx *ctx, velopir_trace_rec *out, size_t cap, size_t *count);

#ifdef __cplusplus
}
#endif
#endif /* VELOPIR_H */
