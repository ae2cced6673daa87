/*
 * grand.h -- C ABI of the GB300 GRAND decoder (arXiv 2405.01808, "GRAND Massive
 * Parallel Decoding Framework for Low Latency in Beyond 5G").
 *
 * The library decodes binary linear codes given by a parity-check matrix H
 * (Def. II.1) from square M-QAM received symbols (Def. II.2). Each frame is
 * demodulated with the paper's likelihood function and its three near-neighbour
 * alternatives per symbol (Def. III.1, III.2), the S' = min(S, L) least
 * reliable symbols are kept (Alg. 2 Steps 2-3), and the test error patterns
 * (TEPs) over them are queried in a fixed canonical order until the first one
 * whose candidate word has a zero syndrome H (y xor e) = 0 (Alg. 2 Steps 4-5),
 * or until a query cap (abandonment, Sec. II). A bit-level GRAND-AB variant
 * (hard decision, TEPs in ascending Hamming weight, Sec. I) is also provided.
 *
 * Canonical order (the paper leaves the order inside the 4^S set open): by the
 * number w of altered symbols, then the colex order of the set of altered
 * reliability ranks (rank 0 = least reliable), then the alternatives read as a
 * base-3 number (h < v < diag) whose least significant digit belongs to the
 * smallest altered rank. A TEP is valid when every chosen alternative exists;
 * invalid TEPs are skipped and not counted. `queries` is the 1-based position
 * of the decoded TEP among valid TEPs, or min(cap, number of valid TEPs) when
 * the frame is abandoned.
 *
 * Conventions for every call:
 *   - Return value 0 (GRAND_OK) or a negative grand_status. No exception
 *     crosses the ABI. Argument errors are detected before any GPU work.
 *   - "device" pointers are CUDA global memory owned by the caller; the
 *     library never frees them. "host" pointers are ordinary CPU memory.
 *     With n_frames == 0 the data pointers may be NULL (nothing is launched).
 *   - Internal scratch comes from a stream-ordered memory pool that the
 *     library creates on each device at its first allocation there and keeps
 *     until the process exits. Its release threshold is UINT64_MAX, so
 *     scratch stays cached between calls instead of being returned to the
 *     system at each synchronisation. The device's default pool (used by
 *     cudaMallocAsync elsewhere in the process) is not touched.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls that
 *     take a stream enqueue asynchronous work on it and return; the caller
 *     synchronises the stream before reading outputs and keeps every buffer
 *     alive until then. Internal scratch is stream-ordered (the pool above).
 *   - Bit packing: a word of N bits is stored in N/32 uint32 words, bit j at
 *     word j >> 5, bit position j & 31 (LSB first).
 *   - A code object is immutable after creation; decodes on different streams
 *     may share it. Destroying it while work on it is in flight is undefined.
 *   - The library keeps per-device state for the life of the process (its
 *     memory pool, the SM count, the no-alloc scratch address, the host-memory calls'
 *     two streams per host thread): a cudaDeviceReset while the library is in
 *     use invalidates it.
 */
#ifndef GRAND_H
#define GRAND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRAND_VERSION 10000 /* 1.0.0 */

typedef enum grand_status {
  GRAND_OK = 0,
  GRAND_E_INVALID = -1,     /* an argument is out of range or NULL */
  GRAND_E_RANK = -2,        /* H does not have full row rank N-K */
  GRAND_E_NOMEM = -3,       /* host or device allocation failed */
  GRAND_E_CUDA = -4,        /* a CUDA runtime call failed */
  GRAND_E_TIMEOUT = -5,     /* a decode's deadline ran out (grand_stream_status) */
  GRAND_E_BUSY = -6,        /* the server cannot admit the request now */
  GRAND_E_UNSUPPORTED = -7, /* valid request outside the built limits */
} grand_status;

/* TEP orders. */
typedef enum grand_order {
  GRAND_ORDER_HAMMING = 0, /* bit-level GRAND-AB: ascending Hamming weight, colex (Sec. I) */
  GRAND_ORDER_QAM_NNE = 1, /* symbol-level, likelihood order of Def. III.1/III.2 (Alg. 2) */
  /* Order variants for comparison with the paper's order:
   * QAM_NEARER  as QAM_NNE, but the horizontal and vertical alternatives of
   *             a symbol swap places when its Q distance to the threshold is
   *             strictly smaller than its I distance (the less reliable axis
   *             is queried first; the diagonal stays last).
   * QAM_NNE5    the five-point nearest-neighbour error model the paper
   *             contrasts with its own (Sec. II, before Cor. III.1): up to
   *             four alternatives per symbol, the neighbouring level on each
   *             side of each axis, in the order toward the received value on
   *             I, toward it on Q, away on I, away on Q; no diagonal. Symbols
   *             are sorted by the same key; O(5^S') patterns. S <= 10. */
  GRAND_ORDER_QAM_NEARER = 2,
  GRAND_ORDER_QAM_NNE5 = 3,
} grand_order;

/* How a TEP's membership H (y ^ e) = 0 is tested (results do not depend on it).
 *   AUTO        syndrome deltas (Alg. 2 Step 4: s(y) xor the H columns a TEP
 *               flips) in the split search of the fused kernels; QAM_NNE5
 *               runs DELTA.
 *   DELTA       syndrome deltas, one TEP per lane and step in canonical
 *               order (no split search); grand_decode_symbols only.
 *   ROW_PARITY  the candidate word y ^ e multiplied by H row by row, each
 *               syndrome bit the parity of (row AND word) -- the product of
 *               Alg. 1 (pMult) evaluated per TEP, stopping at the first odd
 *               row; one TEP per lane; grand_decode_symbols only.
 *   HASH        a decision procedure rather than a test per TEP: the split's A
 *               side (s(y) xor the A deltas) goes into a hash table keyed by
 *               its 32-bit syndrome projection, every B delta is looked up,
 *               and each pair with equal projections is confirmed on the full
 *               syndrome and ranked; the smallest rank is the first hit.
 *               Same outputs as the TEP-by-TEP search (every codeword of the
 *               space is found), O(|A| + |B|) work per frame; stats count only
 *               the confirmed pairs as checks. QAM_NNE / QAM_NEARER, S' <= 12;
 *               not for QAM_NNE5.
 *   FASTEST     grand_autotune / grand_autotune_mixed only: time both
 *               exact choices for the split (AUTO and HASH, identical
 *               outputs) with their launch shapes and write the faster into
 *               params->membership; the decode calls reject it.
 *   SOLVE       no test per TEP: the valid TEPs of a frame (Alg. 2 Step 5
 *               over the S' ranks, at most 4 alternatives each, Def. III.2)
 *               are the flip vectors x over the existing I / Q slots (the
 *               diagonal alternative flips both), and y xor e is a codeword
 *               iff the XOR of the slots' syndrome deltas over x equals s(y):
 *               a linear system over GF(2) with at most 2 S' unknowns. The
 *               preparation solves it by Gaussian elimination; its solutions
 *               are the frame's codewords within the TEP space, and the one of
 *               smallest canonical rank is the first hit (no solution: the
 *               frame abandons with min(valid TEPs, query_cap) queries).
 *               Outputs are those of AUTO (decoded word, query count = the
 *               hit's position in the canonical order, abandon flag); stats
 *               count the ranked solutions as checks. The preparation tests
 *               weights <= 1 first (tiles[2] is not used). Frames whose
 *               solution set has more than 2^8 members go to the TEP search.
 *               QAM_NNE / QAM_NEARER (uniform and uneven batches); not for
 *               QAM_NNE5, HAMMING, the resumable search, the autotuner or
 *               the no-allocation entry point. */
typedef enum grand_membership {
  GRAND_MEMBERSHIP_AUTO = 0,
  GRAND_MEMBERSHIP_DELTA = 1,
  GRAND_MEMBERSHIP_ROW_PARITY = 2,
  GRAND_MEMBERSHIP_HASH = 3,
  GRAND_MEMBERSHIP_FASTEST = 4,
  GRAND_MEMBERSHIP_SOLVE = 5,
} grand_membership;

/* Readings of Def. III.1 for a received value beyond the outermost level. */
typedef enum grand_lik {
  GRAND_LIK_THRESHOLD = 0, /* d = distance to the nearest decision threshold (1 + |A - a|) */
  GRAND_LIK_LITERAL = 1,   /* d = 1 - |A - a| as printed: the ordering key clamps it at 0,
                            * the reported likelihood (rel) uses it unclamped */
} grand_lik;

/* Built limits. */
#define GRAND_N_MIN 32
#define GRAND_N_MAX 1024
#define GRAND_S_MAX 12
#define GRAND_S_MAX_NNE5 10
#define GRAND_AB_WEIGHT_MAX 4

/* Decode parameters.
 *   order       GRAND_ORDER_*.
 *   M           constellation: 2 (BPSK, HAMMING order only), 4, 16, 64, 256, 1024,
 *               4096 (the paper's set, Sec. I contributions and Fig. 4).
 *   S           cut-off (Alg. 2 Step 3), 0..GRAND_S_MAX; S' = min(S, L).
 *   max_weight  HAMMING order: largest number of flipped bits (0..4).
 *   query_cap   abandonment threshold, >= 1 valid queries.
 *   lik_variant GRAND_LIK_*.
 *   tiles       launch shape, 0 = automatic: [0] warps per search CTA (1..8
 *               for explicit splits, 1..4 for the warp-per-frame search and
 *               the hash join), [1] A-side ranks of the search split (1..6; a
 *               nonzero value selects the CTA-per-frame search, 0 the
 *               warp-per-frame search with min(S'/2, 5) ranks on the A side),
 *               [2] number of TEP weights tested by the per-frame preparation
 *               (1..3; automatic: 2), [3] register budget of the search kernel as resident
 *               CTAs of 128 threads per SM (4, 6 or 8; automatic: 4 for the
 *               warp-per-frame search, whose residency shared memory bounds).
 *               Results do not depend on tiles.
 *   membership  GRAND_MEMBERSHIP_*.
 *   deadline_ns device-time budget of the call in nanoseconds, 0 = none
 *               (the watchdog). The budget runs from the first look at the
 *               device clock (%globaltimer) by any warp of the call. A search
 *               warp that fetches a frame after the budget ran out does not
 *               search it: the frame gets abandon = 5, cw = the hard word and
 *               queries = the number of leading valid TEPs already tested
 *               without a hit (those of the preparation stage; 0 for
 *               HAMMING, QAM_NNE5 and the DELTA / ROW_PARITY tests), and the
 *               code's status word is set for grand_stream_status. A frame
 *               whose search has started finishes (at most one frame's search
 *               per warp beyond the budget); frames the preparation resolves
 *               are always decoded. Every other frame's outputs are those of
 *               a call without deadline. */
typedef struct grand_params {
  int32_t order;
  int32_t M;
  int32_t S;
  int32_t max_weight;
  int64_t query_cap;
  int32_t lik_variant;
  int32_t tiles[4];
  int32_t membership;
  int64_t deadline_ns;
} grand_params;

typedef struct grand_code grand_code;

/* One frame of an uneven batch (grand_decode_mixed). Device memory.
 *   code        index into the `codes` array of the call.
 *   M           constellation of this frame (4 .. 4096); L = ceil(N / log2 M).
 *   sym_offset  first received symbol of the frame in the flat symbol array.
 *   cw_offset   first output word of the frame in the flat codeword array. */
typedef struct grand_frame_desc {
  int32_t code;
  int32_t M;
  int64_t sym_offset;
  int64_t cw_offset;
} grand_frame_desc;

/* Per-call counters (optional output of the decode calls; host memory).
 * Requesting them makes the call synchronise its stream before returning.
 *   evaluated_checks  TEP syndrome checks executed on the GPU, including
 *                     speculative ones beyond the first hit.
 *   hard_frames       frames that needed the parallel search stage.
 *   search_useful     valid TEP queries (positions <= the reported query
 *                     count) that fell to the search stage.
 *   prep_ms, search_ms  device time of the preparation and search kernels,
 *                     from CUDA events recorded on the call's stream
 *                     (HAMMING order: prep_ms = 0 and search_ms = the one
 *                     bit-level kernel). */
typedef struct grand_stats {
  uint64_t evaluated_checks;
  uint64_t hard_frames;
  uint64_t search_useful;
  float prep_ms;
  float search_ms;
} grand_stats;

/* Library version (GRAND_VERSION) and a static description of a status. */
int grand_version(void);
const char* grand_status_string(int status);

/* Polar code helper (Def. II.1, Sec. II): G_N = F^{(x)n}; frozen set = the N-K
 * synthetic channels with the largest Bhattacharyya parameter at design SNR
 * `design_snr_db` (E_b/N0, rate-scaled: z0 = exp(-K/N * 10^(snr/10)); ties go
 * to the lower index); H row r = column frozen[r] of G_N, so G_I H^T = 0.
 *   H_out       host, (N-K) rows x (N/32) words, row-major, bit-packed.
 *   frozen_out  host, N-K ascending indices, or NULL.
 * Errors: GRAND_E_INVALID if N is not a power of two in [32, 1024], K < 1,
 * K >= N, or H_out is NULL. Pure host computation. */
int grand_polar_H(int N, int K, double design_snr_db, uint32_t* H_out, int32_t* frozen_out);

/* Create a code from its parity-check matrix (Def. II.1; the membership test
 * of Alg. 2 Step 5 is H x = 0).
 *   H    host, (N-K) x (N/32) words, same layout as grand_polar_H; copied, not
 *        retained. The object keeps a column-packed device copy.
 *   out  receives the new object (host pointer).
 * Errors: GRAND_E_INVALID (N not a power of two in [32, 1024], K < 1,
 * N-K > 512, K >= N, NULL pointers), GRAND_E_RANK (rank H != N-K),
 * GRAND_E_NOMEM, GRAND_E_CUDA. Synchronous on the current device. */
int grand_code_create(const uint32_t* H, int N, int K, grand_code** out);

/* Destroy a code (NULL is a no-op). The caller synchronises first. */
int grand_code_destroy(grand_code* code);

/* N and K of a code (host outputs, either may be NULL). */
int grand_code_info(const grand_code* code, int* N, int* K);

/* Status of the decodes on `code` (the watchdog's read-back): synchronises
 * `stream`, then takes and clears the code's device status word, which every
 * decode call on this code (any stream) sets when a frame was cut by its
 * grand_params.deadline_ns. Returns GRAND_E_TIMEOUT if it was set,
 * GRAND_E_CUDA if the stream reports an error, GRAND_OK otherwise. The word
 * is taken by an atomic exchange on the device, so a flag raised by a
 * concurrent decode on another stream is reported by exactly one read-back;
 * grand_stream_status itself is not called concurrently on one code.
 * Errors: GRAND_E_INVALID (NULL code). */
int grand_stream_status(const grand_code* code, void* stream);

/* Demodulation (Def. III.1, III.2; Alg. 2 Step 1) of n_frames frames of L
 * symbols each.
 *   symbols   device. M >= 4: complex64 (interleaved float32 I, Q) [n_frames][L],
 *             in transmitted units with E_b = 1 per coded bit, d = sqrt(3m/(M-1))
 *             (Eq. 2). M = 2: float32 [n_frames][N] BPSK samples (bit 1 <-> -1).
 *   M         2, 4, 16, 64, 256, 1024 or 4096; L must equal ceil(N / log2 M).
 *   N0        noise spectral density; validated (> 0, finite) but the
 *             likelihood is geometric and does not use it.
 *   lik_variant GRAND_LIK_*.
 *   Outputs (device, any may be NULL; only y is written for M = 2):
 *   hard_idx  uint16 [n_frames][L] = (I level << 8) | Q level, level l has
 *             odd amplitude 2l - (sqrt(M) - 1).
 *   key       uint32 [n_frames][L] = dI^2 + dQ^2 with d the Q8.8 distance of
 *             the received value to its nearest decision threshold (the
 *             fixed-point likelihood; small = unreliable).
 *   nmask     uint8 [n_frames][L]: bit0 h exists, bit1 v exists, bit2 diag
 *             exists, bit3 I direction is +1, bit4 Q direction is +1, bit5
 *             the Q distance is strictly smaller than the I distance (the
 *             vertical alternative is the nearer one), bit7 a coordinate was
 *             not finite (read as 0).
 *   rel       float [n_frames][L] = sqrt(d1^2 + d2^2), Def. III.1, FP32.
 *   y         uint32 [n_frames][N/32] packed hard word: symbol i carries bits
 *             [2m i, 2m i + 2m), I Gray label then Q Gray label, MSB first;
 *             bits >= N are dropped. For M = 2, bit j = [r_j < 0].
 * Errors: GRAND_E_INVALID. Asynchronous on `stream`. */
int grand_demod(const void* symbols, int64_t n_frames, int L, int M, float N0, int lik_variant,
                uint16_t* hard_idx, uint32_t* key, uint8_t* nmask, float* rel, uint32_t* y, int N,
                void* stream);

/* Decode demodulated frames (Alg. 2 Steps 2-5 and Return).
 *   For GRAND_ORDER_QAM_NNE / QAM_NEARER: hard_idx, key, nmask, y as written
 *   by grand_demod with the same M and lik_variant (device). QAM_NNE5 and the
 *   membership tests DELTA / ROW_PARITY: GRAND_E_UNSUPPORTED (use
 *   grand_decode_symbols).
 *   For GRAND_ORDER_HAMMING: only y is read (others may be NULL).
 *   Outputs (device): cw uint32 [n_frames][N/32] decoded word (the hard word
 *   when abandoned); queries uint32 [n_frames]; abandon uint8 [n_frames]:
 *   0 decoded, 1 abandoned (cap reached or TEPs exhausted), 2 not searched
 *   because a received value was not finite, 5 not searched because the
 *   call's deadline (params->deadline_ns) had passed.
 *   stats (host, may be NULL): filled after an internal stream synchronise;
 *   pass NULL to keep the call asynchronous.
 * Errors: GRAND_E_INVALID, GRAND_E_UNSUPPORTED, GRAND_E_NOMEM, GRAND_E_CUDA. */
int grand_decode_batch(const grand_code* code, const grand_params* params, const uint16_t* hard_idx,
                       const uint32_t* key, const uint8_t* nmask, const uint32_t* y, int64_t n_frames,
                       uint32_t* cw, uint32_t* queries, uint8_t* abandon, grand_stats* stats, void* stream);

/* Demodulate and decode in one pass: the per-symbol arrays are not written
 * to memory. symbols as for grand_demod (M = params->M); outputs as for
 * grand_decode_batch. Every QAM order and membership test is accepted here;
 * QAM_NNE5 and membership DELTA / ROW_PARITY run the per-TEP kernel (one
 * warp per frame: demodulation, selection and the canonical walk), whose
 * stats report prep_ms = 0, the walk in search_ms, hard_frames = frames
 * whose first query failed and search_useful = their queries. */
int grand_decode_symbols(const grand_code* code, const grand_params* params, const void* symbols,
                         int64_t n_frames, float N0, uint32_t* cw, uint32_t* queries, uint8_t* abandon,
                         grand_stats* stats, void* stream);

/* Resumable decoding: a frame's TEP search in windows of TEP weights, with
 * the search state (a cursor) kept in device memory between calls.
 *
 * Alg. 2 Step 5 queries the TEPs until the first codeword or the cap. In the
 * canonical order the TEPs come by weight w (altered symbols), so a search
 * that has tested every valid TEP of weight <= w without a hit can continue
 * at weight w + 1 and reach exactly the result of an uninterrupted search:
 * the first hit of the rest of the order is the first hit overall. A cursor
 * holds what the continuation needs: the frame's base syndrome, its S' least
 * reliable symbols (flip positions, existing alternatives) and the weight
 * w_done already tested; GRAND_CURSOR_BYTES bytes, opaque.
 *
 * grand_decode_symbols_resumable: as grand_decode_symbols (orders QAM_NNE and
 * QAM_NEARER, membership AUTO or HASH, automatic split: tiles[1] = 0), but
 * the search of each frame stops after weight_step (>= 1) weight classes
 * beyond those the preparation tested (weights <= 2 with default tiles). A
 * frame with no codeword there, and weights left below the query cap, is
 * suspended: abandon = GRAND_ABANDON_SUSPENDED (6), queries = the valid TEPs
 * tested so far (all of weight <= w_done), cw = its hard word, and its cursor
 * is written to cursors + frame * GRAND_CURSOR_BYTES.
 *   cursors  device, n_frames * GRAND_CURSOR_BYTES bytes, caller-owned; only
 *            the entries of suspended frames are written.
 *   Other frames get their final outputs (decoded, abandoned, 2, 5).
 *
 * grand_decode_resume: the next weight_step weight classes (0: all that are
 * left) of every cursor i in [0, n) whose abandon[i] is 6; cursors whose flag
 * is anything else are skipped, so the same arrays can be passed again until
 * no flag is 6. Cursor i writes queries[i], abandon[i] and, on a hit, flips
 * the decoded bits in cw + i * cw_stride_words (which must hold the frame's
 * hard word, as the first call left it), and its cursor is updated in place
 * when it stays suspended. With the arrays of grand_decode_symbols_resumable
 * (cw_stride_words = N/32) the final outputs equal grand_decode_symbols's
 * for every frame, whatever the steps. params must equal the first call's
 * (S, cap, order); a cursor naming another code, or not describing a search
 * of this code, is marked abandon 3 and not read further.
 * Errors: GRAND_E_INVALID, GRAND_E_UNSUPPORTED (another order or membership
 * test, an explicit split), GRAND_E_NOMEM, GRAND_E_CUDA. Asynchronous. */
#define GRAND_CURSOR_BYTES 144
#define GRAND_ABANDON_SUSPENDED 6
int grand_decode_symbols_resumable(const grand_code* code, const grand_params* params, const void* symbols,
                                   int64_t n_frames, float N0, int32_t weight_step, void* cursors, uint32_t* cw,
                                   uint32_t* queries, uint8_t* abandon, void* stream);
int grand_decode_resume(const grand_code* code, const grand_params* params, void* cursors, int64_t n,
                        int32_t weight_step, uint32_t* cw, int64_t cw_stride_words, uint32_t* queries,
                        uint8_t* abandon, void* stream);

/* Decode an uneven batch: frames of different codes and constellations in
 * one launch sequence (persistent search kernel with a per-frame work queue).
 * The paper decodes one frame of one (N, M) at a time (Alg. 2) and treats
 * frames as independent (Sec. IV, no interleaving across codewords); batching
 * frames of every N in {32..1024} and M of its set (Sec. I, Fig. 4 setup) into
 * one launch is this library's own pattern for filling a GPU, with per-frame
 * results equal to Alg. 2's for that frame alone.
 *   codes      host array of n_codes code pointers.
 *   desc       device array of n_frames grand_frame_desc.
 *   symbols    device complex64, flat, n_symbols entries; frame f starts at
 *              desc[f].sym_offset.
 *   cw         device uint32, flat, n_cw_words entries; frame f starts at
 *              desc[f].cw_offset.
 *   params     order GRAND_ORDER_QAM_NNE or QAM_NEARER with membership
 *              AUTO, HASH or SOLVE; params->M is ignored (each frame has its own);
 *              S' = min(params->S, L) per frame.
 * Errors as for grand_decode_batch. A descriptor with an unknown code, an
 * unsupported M or a range outside the arrays is not decoded: its abandon
 * flag is 3 and its queries 0 (checked on the device). */
int grand_decode_mixed(const grand_code* const* codes, int n_codes, const grand_params* params,
                       const grand_frame_desc* desc, int64_t n_frames, const void* symbols, int64_t n_symbols,
                       float N0, uint32_t* cw, int64_t n_cw_words, uint32_t* queries, uint8_t* abandon,
                       grand_stats* stats, void* stream);

/* Plans (no counterpart in the paper, whose Prop. III.1 counts circuit clock
 * cycles: on a GPU the fixed cost per call is the launch sequence, and a graph
 * replays it with one launch): one decode call captured into a CUDA graph, replayed by
 * grand_plan_launch on any stream with the buffers given at creation (the
 * caller refills the inputs between launches; outputs are overwritten). The
 * captured sequence is the same as the direct call's (counter reset,
 * preparation kernel, persistent search kernel with its work queue, scratch as
 * graph memory nodes), so results are identical. Creation runs the call once
 * eagerly on a private stream and synchronises it; it must not be called
 * while the calling thread captures a stream. A plan's launches must not
 * overlap each other in time (they share the buffers); the caller orders them.
 *   grand_plan_symbols: arguments as grand_decode_symbols (n_frames >= 1).
 *   grand_plan_mixed:   arguments as grand_decode_mixed; the code table is
 *                       copied into the plan (codes must outlive the plan).
 * Errors: as the direct calls, plus GRAND_E_CUDA if capture fails. */
typedef struct grand_plan grand_plan;
int grand_plan_symbols(const grand_code* code, const grand_params* params, const void* symbols, int64_t n_frames,
                       float N0, uint32_t* cw, uint32_t* queries, uint8_t* abandon, grand_plan** out);
int grand_plan_mixed(const grand_code* const* codes, int n_codes, const grand_params* params,
                     const grand_frame_desc* desc, int64_t n_frames, const void* symbols, int64_t n_symbols,
                     float N0, uint32_t* cw, int64_t n_cw_words, uint32_t* queries, uint8_t* abandon,
                     grand_plan** out);
int grand_plan_launch(grand_plan* plan, void* stream);
int grand_plan_destroy(grand_plan* plan);

/* Launch-shape autotuner (no counterpart in the paper: its parallel design
 * fixes 4^S instances, Prop. III.1, where a GPU must choose how many frames,
 * TEPs and table slices share an SM). Times every candidate `tiles` setting (preparation
 * weights, search register budget, and for S' > 10 the warps per CTA) on the
 * given sample with CUDA events (median of 3 runs after one untimed run) and
 * writes the fastest into params->tiles. With params->membership =
 * GRAND_MEMBERSHIP_FASTEST the candidates also span the membership test (the
 * TEP-by-TEP split search and the hash join, with the hash join's own launch
 * shapes) and the chosen one is written into params->membership. Results
 * never depend on the choice.
 *   cache_path  host path of a text cache (NULL: no cache). Lines are
 *               "key t0 t1 t2 t3 ms membership"; the key holds the GPU name
 *               and the workload (N, K, M, S, cap, likelihood variant, the
 *               membership asked for; the codes of a mixed batch). A cached
 *               key is used without timing.
 *   out         host, may be NULL: best time, candidates tried, cache hit,
 *               the membership test chosen.
 * The sample buffers are device memory; the tuner allocates its own outputs
 * (cudaMalloc) and synchronises `stream`. Errors: as the decode calls. */
typedef struct grand_tune_result {
  float best_ms;
  int32_t candidates;
  int32_t from_cache;
  int32_t membership;
} grand_tune_result;
int grand_autotune(const grand_code* code, grand_params* params, const void* symbols, int64_t n_frames, float N0,
                   const char* cache_path, void* stream, grand_tune_result* out);
int grand_autotune_mixed(const grand_code* const* codes, int n_codes, grand_params* params,
                         const grand_frame_desc* desc, int64_t n_frames, const void* symbols, int64_t n_symbols,
                         float N0, int64_t n_cw_words, const char* cache_path, void* stream, grand_tune_result* out);

/* Serving loop (continuous batching of decode requests). The paper's target
 * is per-frame latency for 5G and beyond (Sec. I: over-the-air latency under
 * 1 ms); it decodes one frame per invocation of its parallel circuit. This
 * loop is the library's way to meet a latency bound while frames arrive at
 * millions per second: requests join the next batch on a free stream instead
 * of waiting for a whole batch. A request is one
 * frame of any of the server's codes and any constellation. Submit admits
 * requests while a slot is free and the device memory budget allows (bytes
 * per request: 8 L received symbols + 144 hand-off record + N/8 + 5
 * outputs); admitted requests keep their received word resident on the
 * device (a device ring mirrored from pinned host memory) until they
 * complete. A launcher thread issues all admitted, not yet launched requests
 * as one uneven batch on the first idle stream (the grand_decode_mixed
 * sequence), so requests arriving while batches run are decoded concurrently
 * on other streams; a harvester thread collects finished batches. Results
 * are exactly those of grand_decode_mixed / grand_decode_symbols for the same
 * frame, whatever the batch it landed in.
 *   codes             host array of n_codes code pointers (borrowed; they must
 *                     outlive the server).
 *   params            order GRAND_ORDER_QAM_NNE or QAM_NEARER, membership
 *                     AUTO, HASH or SOLVE (SOLVE without resume_weight_step);
 *                     M comes with each request.
 *   max_slots         admitted requests resident at once.
 *   max_device_bytes  memory budget of the resident request state; the
 *                     symbol ring holds max_device_bytes / 8 symbols.
 *   max_batch         frames per launch (0: max_slots).
 *   n_streams         batches in flight at once (1..16).
 *   resume_weight_step  0: each frame is searched whole inside its batch.
 *                     k > 0: a batch searches each frame's TEPs only up to k
 *                     weight classes beyond the preparation's (the weight
 *                     windows of grand_decode_symbols_resumable, tiles[1] = 0).
 *                     The batch's other frames are reported as soon as that
 *                     launch ends and its stream takes the next batch; the
 *                     frames left without a codeword continue -- every
 *                     remaining weight -- from their device-resident cursors
 *                     on a separate stream, and are reported when done. Every
 *                     result equals the uninterrupted search's. The server
 *                     then holds 4 x n_streams buffer sets (a batch keeps
 *                     its set until its last frame is reported).
 *   params.deadline_ns, when nonzero, is the budget of each batch launch (and
 *   of each continuation). */
typedef struct grand_server_cfg {
  const grand_code* const* codes;
  int32_t n_codes;
  grand_params params;
  float N0;
  int32_t max_slots;
  int64_t max_device_bytes;
  int32_t max_batch;
  int32_t n_streams;
  int32_t resume_weight_step;
} grand_server_cfg;

/* One decode request. symbols: host complex64 [L], L = ceil(N / log2 M) of the
 * request's code, copied during submit. arrival_ns: arrival time on the
 * grand_clock_ns() clock (0: the submit time); latency = done - arrival. */
typedef struct grand_request {
  int32_t code;
  int32_t M;
  const void* symbols;
  uint64_t tag;
  int64_t arrival_ns;
} grand_request;

/* One completed request: decoded word (first N/32 words of cw), query count,
 * abandon flag (as grand_decode_batch; 4 = the batch failed on the device),
 * continued = 1 when the frame's search went on after its batch was reported
 * (resume_weight_step > 0), else 0. */
typedef struct grand_result {
  uint64_t tag;
  int64_t arrival_ns;
  int64_t done_ns;
  uint32_t queries;
  uint8_t abandon;
  uint8_t continued;
  uint8_t pad[2];
  uint32_t cw[GRAND_N_MAX / 32];
} grand_result;

/* Counters of a server. batch_service_ns: sum over batches of (completion seen
 * - launch start); launch_ns: host time spent issuing batches (copies, decode
 * call, event). long_frames: frames continued after their batch's first
 * launch (resume_weight_step > 0); resume_launches: continuation launches;
 * long_live: frames being continued now. */
typedef struct grand_server_stats {
  int64_t admitted, rejected, completed, batches, batched_frames, max_inflight_batches, errors;
  int64_t live_slots, live_bytes, pending, inflight_batches;
  int64_t batch_service_ns, max_batch_service_ns, launch_ns, max_launch_ns;
  int64_t long_frames, resume_launches, long_live;
} grand_server_stats;

typedef struct grand_server grand_server;

/* Host monotonic clock of the server, nanoseconds. */
int64_t grand_clock_ns(void);
/* Create a server on the current device (allocates the ring, per-stream
 * buffers, streams, and starts the launcher and harvester threads). */
int grand_server_create(const grand_server_cfg* cfg, grand_server** out);
/* Admit requests in order until one does not fit; *n_admitted of them were
 * taken. Returns GRAND_OK if at least one was admitted (or n == 0),
 * GRAND_E_BUSY if none fits now, GRAND_E_INVALID on a malformed request
 * (the requests before it stay admitted). Thread-safe. */
int grand_server_submit(grand_server* srv, const grand_request* reqs, int n, int* n_admitted);
/* Move up to max completed results into out (host); *n of them. Thread-safe. */
int grand_server_poll(grand_server* srv, grand_result* out, int max, int* n);
/* Wait until every admitted request completed; GRAND_E_TIMEOUT after
 * timeout_ns (results stay queued for poll). */
int grand_server_drain(grand_server* srv, int64_t timeout_ns);
int grand_server_get_stats(grand_server* srv, grand_server_stats* out);
/* Drain (bounded: 10 s), stop the threads and free everything. */
int grand_server_destroy(grand_server* srv);

/* grand_decode_symbols without any allocation (the paper has no counterpart:
 * this is a deployment convenience). For callers that are not allowed to
 * allocate device memory once they are running -- for example a real-time
 * receiver pipeline that reserves all memory at start-up, or code running
 * where the stream-ordered allocator is unavailable or would break a latency
 * budget. Same inputs, outputs and results as grand_decode_symbols with the
 * same params; the caller still provides every input and output buffer.
 *   - Internal scratch is a fixed array of about 2.4 MB in the library's
 *     device memory, present on every GPU that loads the library until the
 *     process exits. It holds at most GRAND_NOALLOC_MAX_FRAMES frames: larger
 *     n_frames is rejected with GRAND_E_UNSUPPORTED before any GPU work.
 *   - Only GRAND_ORDER_QAM_NNE with membership AUTO; no statistics output.
 *   - The first call on a device looks up the array's device address (a
 *     one-time set-up); make that first call before any stream capture.
 *   - Every call on a device shares the one array and resets its counters
 *     first: calls whose GPU work overlaps in time (different streams, or
 *     different host threads) race and give wrong results. Serialise them.
 * Errors: GRAND_E_INVALID, GRAND_E_UNSUPPORTED, GRAND_E_CUDA. */
#define GRAND_NOALLOC_MAX_FRAMES 16384
int grand_decode_symbols_noalloc(const grand_code* code, const grand_params* params, const void* symbols,
                                 int64_t n_frames, float N0, uint32_t* cw, uint32_t* queries, uint8_t* abandon,
                                 void* stream);

/* Decode frames held in host memory (the decode of grand_decode_symbols with
 * the transfers included and overlapped). The batch is cut into chunks of
 * chunk_frames frames (0: a quarter of the batch, at least 65,536) that
 * alternate between two internal streams with their own device buffers; on
 * each, a chunk's symbols are copied to the device, decoded and its results
 * copied back, so that the copies of one chunk run while another is decoded.
 *   h_symbols  host, as `symbols` of grand_decode_symbols (complex64 [n][L],
 *              or float32 [n][N] for the HAMMING order).
 *   h_cw, h_queries, h_abandon  host outputs, as for grand_decode_symbols.
 *   Host buffers should be page-locked (cudaHostAlloc / cudaHostRegister):
 *   copies from pageable memory are staged by the CUDA driver and overlap less.
 *   stream     the work starts after what is queued on it; on return every
 *              result is in host memory and `stream` is ordered after the
 *              pipeline (the call is synchronous).
 * Each chunk is one decode call: a deadline (params->deadline_ns) applies per
 * chunk. Errors: as grand_decode_symbols (arguments checked before any device
 * work), GRAND_E_NOMEM, GRAND_E_CUDA. */
int grand_decode_symbols_host(const grand_code* code, const grand_params* params, const void* h_symbols,
                              int64_t n_frames, float N0, uint32_t* h_cw, uint32_t* h_queries, uint8_t* h_abandon,
                              int64_t chunk_frames, void* stream);

/* Decode an uneven batch held in host memory (grand_decode_mixed with the
 * transfers included and overlapped the same way).
 *   h_desc     host array of n_frames descriptors (offsets into h_symbols and
 *              h_cw, as for grand_decode_mixed).
 *   h_symbols  host complex64, n_symbols entries; h_cw host, n_cw_words words;
 *              h_queries, h_abandon host, n_frames entries. Every host buffer,
 *              the descriptors included, should be page-locked: a copy from
 *              pageable memory holds the calling thread until it is staged.
 * Chunks are runs of consecutive frames; they need the frames packed in
 * increasing order (each frame's symbols and output words after the previous
 * frame's, inside the arrays). Any other layout is decoded as one chunk over
 * the whole arrays (no overlap). A chunk's descriptors are made relative to
 * its own ranges on the device; a descriptor that is invalid there is
 * reported as by grand_decode_mixed (abandon 3). Arguments are checked first
 * (by a call of grand_decode_mixed without frames). Errors: as
 * grand_decode_mixed, GRAND_E_NOMEM, GRAND_E_CUDA. */
int grand_decode_mixed_host(const grand_code* const* codes, int n_codes, const grand_params* params,
                            const grand_frame_desc* h_desc, int64_t n_frames, const void* h_symbols, int64_t n_symbols,
                            float N0, uint32_t* h_cw, int64_t n_cw_words, uint32_t* h_queries, uint8_t* h_abandon,
                            int64_t chunk_frames, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GRAND_H */
