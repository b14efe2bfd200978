/*
 * sfa.h -- C ABI of the GB300 (sm_103a) simultaneous-finite-automaton matcher.
 *
 * The library runs the data-parallel computation of a D-SFA (Sin'ya,
 * Matsuzaki, Sassa, "Simultaneous Finite Automata: An Efficient Data-Parallel
 * Model for Regular Expression Matching", ICPP 2013) on one GPU:
 *
 *   - sfa_compile    builds the D-SFA of a DFA on the host (Alg. 4, with the
 *                    DFA simplification of Sect. V-A) and uploads its tables;
 *   - sfa_match*     split a text into chunks, run the SFA on every chunk from
 *                    the identity state f_I (Alg. 5), combine the per-chunk
 *                    mappings by reverse composition (Lemma 1, Theorem 3) and
 *                    count the prefixes that end in a final state.
 *
 * Semantics of every match call, for a DFA (Q, Sigma, delta, {q0}, F) and a
 * text w = w_1 .. w_n (Sect. II-B, Alg. 2):
 *   final_state  = delta^(q0, w)            (q0 when n = 0)
 *   accept_final = 1 iff final_state is in F
 *   count        = #{ i in 1..n : delta^(q0, w_1..w_i) in F }
 * (the empty prefix is not counted; overlapping occurrences all count).
 * All results are integers and exact.
 *
 * Conventions
 *   - State numbers in and out of the library are the caller's (0..nq-1).
 *   - Pointers named d_* are device pointers of the current device; h_* and
 *     unprefixed array arguments are host pointers.
 *   - Match calls only enqueue work on `stream` and return; results are valid
 *     once the stream has reached that point.  Inputs must stay alive and
 *     unmodified until then.  Exception: sfa_match_host synchronises.
 *   - Every function returns SFA_OK (0) or a negative SFA_ERR_* code and
 *     never throws; sfa_strerror gives a message.
 *   - A handle's scratch memory is shared by its match calls: calls on one
 *     handle must not overlap on the GPU (use one stream per handle, or one
 *     handle per stream).
 */
#ifndef SFA_H
#define SFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The CUDA runtime's cudaStream_t (NULL = the legacy default stream). */
typedef struct CUstream_st *sfa_stream_t;

typedef struct sfa_handle *sfa_handle_t;
typedef struct sfa_batch *sfa_batch_t;

/* ---- error codes ------------------------------------------------------- */
#define SFA_OK               0
#define SFA_ERR_INVALID     -1  /* bad argument: DFA out of range, NULL pointer, size */
#define SFA_ERR_UNSUPPORTED -2  /* valid but outside the library's limits (e.g. nq > 4095) */
#define SFA_ERR_OOM         -3  /* host or device allocation failed */
#define SFA_ERR_CUDA        -4  /* a CUDA runtime call failed */
#define SFA_ERR_TIMEOUT     -5  /* a device-side bounded wait gave up (see sfa_result.status) */
#define SFA_ERR_NO_DEVICE   -6  /* no CUDA device is usable */
#define SFA_ERR_HOST_ONLY   -7  /* the handle was compiled with SFA_COMPILE_HOST_ONLY */
#define SFA_ERR_SCRATCH_LIMIT -8 /* sfa_match_noalloc: the text needs more scratch than
                                    the fixed buffer holds */

/* ---- result of one text (16 bytes, written to device memory) ----------- */
typedef struct {
    uint32_t final_state;   /* delta^(q0, w), caller's numbering */
    uint8_t accept_final;   /* 1 iff final_state is final */
    uint8_t status;         /* 0 = valid; SFA_STATUS_TIMEOUT = a device-side
                               wait gave up and the other fields are invalid */
    uint16_t reserved;
    uint64_t count;         /* accepting prefixes, see above */
} sfa_result;

#define SFA_STATUS_OK      0
#define SFA_STATUS_TIMEOUT 1

/* ---- compile ------------------------------------------------------------ */
#define SFA_MODE_AUTO 0     /* D-SFA if it stays within cap_states, else simulation */
#define SFA_MODE_SFA  1     /* always the D-SFA (fails with UNSUPPORTED past the cap) */
#define SFA_MODE_SIM  2     /* always the simulation path of Alg. 3 */

#define SFA_COMPILE_HOST_ONLY 1u  /* build the tables on the host only; no device
                                     memory, match calls fail with SFA_ERR_HOST_ONLY */
#define SFA_COMPILE_NO_BANK_TUNE 2u  /* keep the breadth-first numbering of the kept
                                     states (final states last) instead of choosing the
                                     ids against shared-memory bank conflicts */

typedef struct {
    uint32_t cap_states;    /* max non-constant D-SFA states; 0 = 65536 */
    int32_t force_mode;     /* SFA_MODE_* */
    uint32_t flags;         /* SFA_COMPILE_* */
    uint32_t reserved;
} sfa_compile_opts;

/*
 * sfa_compile -- Alg. 4 (correspondence construction), Sect. V-A.
 *   delta   host, int32[nq * 256], row-major: delta[q*256 + b] is the state
 *           after reading byte b in state q; every entry in [0, nq)
 *   nq      1..4095 states
 *   q0      initial state, [0, nq)
 *   accept  host, uint8[nq]: nonzero = final state
 *   opts    NULL for defaults
 *   out     receives the handle (owns host and device tables)
 * Synchronous.  Device tables go to the current device.  The D-SFA is built
 * over the states reachable from q0 and over byte classes (bytes whose
 * columns of delta are equal); when it has more than cap_states
 * non-constant mappings the handle uses the simulation path (Alg. 3), which
 * is not an error.  The kept states are numbered breadth first from q0,
 * final states last; unless SFA_COMPILE_NO_BANK_TUNE is set, the ids within
 * each kind are then chosen by a local search that lowers the modelled
 * shared-memory bank conflicts of the kernel's DFA-row lookups (lanes run
 * over bytes drawn uniformly from the bytes that can change a state; about
 * 20-40 ms of host time for 50-160 states).  Numbering never changes a result.
 * With more than 256 reachable states (up to 4095) the ids are 16-bit, the
 * DFA rows are indexed by byte class, and point mappings {s -> p, every other
 * state -> z} (z an absorbing non-final state) are not stored: the matcher
 * follows p through the DFA rows, so only the other non-constant mappings
 * count against cap_states.  Such handles have no simulation path.
 * Errors: INVALID (range), UNSUPPORTED (nq > 4095, SFA_MODE_SFA forced past
 * the cap, more than 256 reachable states past the cap or with
 * SFA_MODE_SIM), OOM, CUDA, NO_DEVICE.  Every DFA of 1..256 states compiles
 * in SFA_MODE_AUTO (simulation vectors cover up to 256 reachable states).
 */
int sfa_compile(const int32_t *delta, int32_t nq, int32_t q0, const uint8_t *accept,
                const sfa_compile_opts *opts, sfa_handle_t *out);

/*
 * sfa_compile_sample -- sfa_compile with the bank-conflict model of the
 * state numbering driven by a sample of the texts to come instead of
 * uniform bytes (the lanes of the model start at pseudo-random offsets of
 * the sample).  The paper has no counterpart: it only changes where DFA rows
 * sit in shared memory, never a result.
 *   sample      host bytes, read during the call only (not kept)
 *   sample_len  bytes of sample; below 1456 the uniform model is used
 * Ignored with SFA_COMPILE_NO_BANK_TUNE.  Errors: as sfa_compile, and
 * INVALID for sample == NULL with sample_len > 0.
 */
int sfa_compile_sample(const int32_t *delta, int32_t nq, int32_t q0, const uint8_t *accept,
                       const sfa_compile_opts *opts, const uint8_t *sample, uint64_t sample_len,
                       sfa_handle_t *out);

/* sfa_destroy -- frees a handle (NULL is fine).  The caller guarantees that
 * no work using it is in flight. */
void sfa_destroy(sfa_handle_t h);

/* ---- information -------------------------------------------------------- */
typedef struct {
    uint32_t mode;            /* SFA_MODE_SFA or SFA_MODE_SIM */
    uint32_t nq;              /* states given to sfa_compile */
    uint32_t n_reachable;     /* states reachable from q0 (the ones kept) */
    uint32_t n_accepting;     /* reachable final states */
    uint32_t ncls;            /* byte classes */
    uint32_t on_device;       /* 1 if device tables exist */
    uint64_t n_sfa_states;    /* |Q_s| (reachable from f_I); 0 in SIM mode */
    uint64_t n_nonconst;      /* of which non-constant mappings */
    uint64_t table_bytes;     /* device bytes of all tables */
    double compile_seconds;   /* host construction time */
    uint64_t n_stored;        /* non-constant mappings stored as rows; the others
                                 (point mappings of automata with more than 256
                                 reachable states) are followed implicitly */
    uint32_t id_bits;         /* 8: byte state ids (up to 256 reachable states);
                                 16: up to 4095 */
    uint32_t placement;       /* SFA_PLACE_* bits: where the kernel reads its tables */
} sfa_info_t;

#define SFA_PLACE_SMEM_DFA          1u  /* DFA rows (256 byte columns) in shared memory */
#define SFA_PLACE_SMEM_DFA_CLASSES  2u  /* 16-bit DFA rows over byte classes in shared memory */
#define SFA_PLACE_GLOBAL_NC         4u  /* non-constant D-SFA rows in global memory (L1/L2) */
#define SFA_PLACE_SMEM_VECTORS      8u  /* simulation vectors of 128/256 entries in shared memory */

/* sfa_info -- fills *out.  Thm. 2 bounds n_sfa_states by n_reachable^n_reachable.
 * n_sfa_states counts every D-SFA state reachable from f_I (stored, implicit
 * point mappings, constants); n_nonconst the non-constant ones among them. */
int sfa_info(sfa_handle_t h, sfa_info_t *out);

/* sfa_export -- copies one host table of the handle, for inspection and tests.
 *   which: SFA_TABLE_CLASS  uint8[256]            class of each byte
 *          SFA_TABLE_DFA    uint8[nr * 256]       renumbered DFA, row = state
 *          SFA_TABLE_NC     uint32[n_nc * ncls]   non-constant D-SFA rows:
 *                           next id in bits 0..29, class of next in 30..31
 *                           (0 no state final, 1 all final, 2 mixed)
 *          SFA_TABLE_MAPS   uint8[n_nc * nr]      mapping of each non-constant state
 *          SFA_TABLE_ORIG   int32[nr]             caller's id of each kept state
 *   Kept states are renumbered so that the final ones come last; D-SFA id
 *   c < nr is the constant mapping onto state c, id nr + k the k-th
 *   non-constant mapping in discovery order (k = 0 is f_I when nr > 1).
 *   Handles with 16-bit ids (more than 256 reachable states) have empty DFA
 *   and MAPS tables and export CDFA16 and MAPS16 instead; their NC entries
 *   that lead to a point mapping {s -> p, all other states -> the sink} hold
 *   1 << 29 | s << 12 | p instead of an id, and those that lead to a
 *   set-point mapping {q in S -> p, all other states -> the sink} (S of two
 *   or more states) hold 1 << 29 | 1 << 28 | sid << 12 | p, S being row sid
 *   of SFA_TABLE_SETS.
 *   Writes min(bytes, table size); returns the table size in *size_out.
 */
#define SFA_TABLE_CLASS 0
#define SFA_TABLE_DFA   1
#define SFA_TABLE_NC    2
#define SFA_TABLE_MAPS  3
#define SFA_TABLE_ORIG  4
#define SFA_TABLE_CDFA16 5  /* uint16[nr * ncls]  kept DFA over classes (16-bit ids only) */
#define SFA_TABLE_MAPS16 6  /* uint16[n_stored * nr] stored mappings (16-bit ids only) */
#define SFA_TABLE_SETS   7  /* uint32[n_sets * ((nr + 31) / 32)] source sets of the set-point
                               mappings, bit q of set s at word s * ((nr + 31) / 32) + q / 32
                               (16-bit ids only) */
int sfa_export(sfa_handle_t h, int32_t which, void *dst, size_t bytes, size_t *size_out);

/* sfa_strerror -- static message for an SFA_* code. */
const char *sfa_strerror(int code);

/* ---- launch shape (all fields optional: 0 = automatic) ------------------ */
#define SFA_DEBUG_SKIP_PUBLISH 1u  /* test knob: tile 1 never publishes its look-back
                                      descriptor, so its successor's bounded wait runs out */
/* What a tile of the decoupled look-back is (Sect. IV's combine over chunks):
 *   SFA_TILING_WARP  one warp's 32 consecutive chunks.  Every warp takes its
 *                    own tiles, publishes its own descriptor and finishes its
 *                    own tiles; single texts with chains = 1 only.
 *   SFA_TILING_CTA   one CTA's block_threads * chains consecutive chunks,
 *                    combined in shared memory before the look-back.  With
 *                    automatic chunks and two CTAs per SM, a long text is cut
 *                    into two levels of different chunk lengths: one tile per
 *                    SM for the CTA that starts first there (the faster one)
 *                    and a shorter one for the other.
 *   SFA_TILING_AUTO  CTA tiles.  Batches always take CTA tiles
 *                    (SFA_TILING_WARP: unsupported). */
#define SFA_TILING_AUTO 0u
#define SFA_TILING_CTA  1u
#define SFA_TILING_WARP 2u

typedef struct {
    uint32_t chunk_bytes;     /* bytes per chunk (any value >= 1; 0 = automatic) */
    uint32_t block_threads;   /* 128, 256, 512, or 1024 with chains = 1 (0 = automatic) */
    uint32_t chains;          /* chunks per thread: 1, 2 or 4 (0 = automatic) */
    uint32_t max_ctas;        /* cap on resident CTAs (0 = all that fit) */
    uint32_t forced_chunks;   /* >0: split the text into exactly this many chunks of
                                 equal length (+-1 byte) instead of chunk_bytes */
    uint32_t timeout_us;      /* bound on each device-side wait (0 = 2 s) */
    uint32_t debug_flags;     /* SFA_DEBUG_* */
    uint32_t tiling;          /* SFA_TILING_* */
} sfa_launch_opts;

/* ---- matching ------------------------------------------------------------ */

/*
 * sfa_match -- Alg. 5 on the GPU for one device-resident text.
 *   d_text  device, n bytes (any alignment); may be NULL when n = 0
 *   n       text length, up to 2^40
 *   d_out   device, one sfa_result
 * The text is split into chunks; every chunk is run from f_I; the chunk
 * mappings are combined by warp, block and grid (decoupled look-back) scans
 * of reverse compositions (Lemma 1, Theorem 3); a second pass over each
 * chunk's prefix before its last "mixed" position counts final states.
 * With no launch options, a D-SFA handle with byte state ids matches a text
 * of up to 1 MiB with the short-text kernel instead: one CTA (up to 16 KiB)
 * or a thread-block cluster of up to 16 CTAs whose aggregates meet in
 * distributed shared memory; no scratch and no look-back (a cluster size the
 * device cannot hold resident falls back to the persistent kernel).
 * May grow the handle's scratch (cudaMalloc) when n exceeds all previous calls.
 */
int sfa_match(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out,
              sfa_stream_t stream);

/* sfa_match_ex -- sfa_match with an explicit launch shape (opts may be NULL). */
int sfa_match_ex(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out,
                 sfa_stream_t stream, const sfa_launch_opts *opts);

/*
 * sfa_match_continue -- streaming form of Lemma 1: *d_inout holds the result
 * for a text u (as written by a previous match call on this handle); on
 * completion it holds the result for u w, where w = d_text[0..n).  So a long
 * text can be matched piece by piece with identical results.
 */
int sfa_match_continue(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_inout,
                       sfa_stream_t stream, const sfa_launch_opts *opts);

/*
 * sfa_match_map -- the mapping of a text slice (Lemma 1, Theorem 3).  For a
 * slice w of a longer text: d_map[q] = delta^(q, w) for every state q that is
 * reachable from q0 (caller ids), -1 for the states that are not.  With
 * sfa_match_continue this splits one text over several processes or
 * devices: each part computes its slice's mapping; the mappings of the
 * parts before it, applied in order to q0, give its entering state s; a
 * result record {final_state = s, count = 0} passed to sfa_match_continue
 * then gives its count and its final state (Theorem 3: the results do not
 * depend on where the text was cut).
 *   d_text, n  the slice (device, any alignment; may be NULL when n = 0)
 *   d_out      device, one sfa_result: the slice matched from q0, as sfa_match
 *   d_map      device, int32[nq] (nq as given to sfa_compile)
 *   opts       launch shape (NULL = automatic); SFA_TILING_WARP is INVALID
 *              (the mapping is composed from CTA-tile aggregates)
 * Enqueues the matching kernel, in which every tile also leaves its mapping
 * in scratch, and one small kernel that composes them, both on `stream`.
 * Errors as sfa_match_ex, and INVALID for d_map == NULL.
 */
int sfa_match_map(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out, int32_t *d_map,
                  sfa_stream_t stream, const sfa_launch_opts *opts);

/*
 * sfa_match_host -- end-to-end form: host text in, host result out.
 *   h_text  host, n bytes (pinned memory gives full copy bandwidth)
 *   h_out   host, one sfa_result
 * Copies the text to the device in pieces on a second stream, overlapping
 * each copy with the matching of the previous piece (sfa_match_continue),
 * and synchronises before returning.  Uses handle-owned staging buffers.
 * A text of up to 256 KiB in pinned host memory the device can read
 * (mapped, e.g. from cudaHostAlloc) is matched in place, without a staging
 * copy, when the automatic shape applies (no launch options set); its result
 * goes to a handle-owned mapped pinned record (allocated on the first such
 * call) and is copied to h_out after the synchronisation.
 */
int sfa_match_host(sfa_handle_t h, const uint8_t *h_text, uint64_t n, sfa_result *h_out,
                   sfa_stream_t stream, const sfa_launch_opts *opts);

/*
 * sfa_match_noalloc -- sfa_match for callers that must not allocate device
 * memory while they match.  Examples: a plugin running inside a host program
 * that owns all device memory through its own pool and forbids outside
 * cudaMalloc calls, or a latency-bound loop that cannot afford cudaMalloc /
 * cudaFree, which may block the host and synchronise the device.
 * (The paper has no counterpart; this is an interface for such callers.)
 *
 * It runs the same D-SFA kernel as sfa_match.  The kernel's scratch (look-back
 * descriptors, tile aggregates, the per-text record) lives in a fixed
 * SFA_NOALLOC_SCRATCH_BYTES array compiled into the library instead of in
 * handle-owned memory; every GPU that loads the library holds one copy until
 * the process exits.  The caller still passes the text and the result buffer.
 *   - No cudaMalloc, cudaFree or other allocating call is made.  Every call
 *     looks up the array's device address on the current device
 *     (cudaGetSymbolAddress, which allocates nothing), so no address taken
 *     before a cudaDeviceReset is used after it; the first call on a device may load the
 *     library's device code there, so make it before any stream capture.
 *   - The handle must be in SFA mode (simulation handles: SFA_ERR_UNSUPPORTED),
 *     have device tables (else SFA_ERR_HOST_ONLY) and live on the current
 *     device (else SFA_ERR_INVALID).  Every refusal is returned before any
 *     work is enqueued and before the array's address is looked up.
 *   - A text whose scratch would not fit is rejected with
 *     SFA_ERR_SCRATCH_LIMIT before any work is enqueued.  The scratch is about
 *     8 + nr bytes per tile (nr = reachable states), and the automatic chunk
 *     length gives at most one tile per resident CTA, so every text up to the
 *     2^40-byte maximum fits (under 100 KB for nr = 256).
 *   - All calls share the one array, and it keeps the last call's contents:
 *     each call clears the parts that must start at zero.  Calls that overlap
 *     on the GPU (two streams, two threads, two handles) race on the array and
 *     give wrong results; issue them on one stream, one after another.
 */
#define SFA_NOALLOC_SCRATCH_BYTES (4u << 20)
int sfa_match_noalloc(sfa_handle_t h, const uint8_t *d_text, uint64_t n, sfa_result *d_out,
                      sfa_stream_t stream);

/* ---- batches ------------------------------------------------------------- */

/*
 * sfa_batch_create -- plans one persistent launch over k texts, each matched
 * with its own automaton (Theorem 3 applied per text: every text gets its own
 * look-back chain of tiles).
 *   hs       host, k handles (all compiled on the current device).  The
 *            texts of simulation-mode handles run in one more persistent
 *            launch per vector size (16, 32, 64, 128 or 256 entries); texts
 *            of handles with 16-bit state ids take per-text launches
 *   d_texts  host array of k device pointers
 *   lens     host, k lengths
 *   opts     launch shape (NULL = automatic)
 * The work list (texts sorted by automaton, tiles in text order) and the
 * scratch are allocated and uploaded here, synchronously; launches of the
 * plan allocate nothing and can be captured in a CUDA graph.
 */
int sfa_batch_create(const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens,
                     int32_t k, const sfa_launch_opts *opts, sfa_batch_t *out);

/*
 * sfa_batch_reserve -- a plan with capacity but no work list yet, for loops
 * that launch a different set of texts each time (serving).
 *   max_texts  texts per launch
 *   max_tiles  tiles per launch; a text of n bytes takes at most
 *              1 + n / (threads * chains * chunk_bytes) tiles
 *   nr_max     largest reachable-state count of the automata to be used
 *   opts       launch shape; chunk_bytes fixes the chunk length (0 = 1024)
 * Allocates device memory and pinned staging once (synchronous).  Its
 * launches read the tile count on the device, so they stay valid (and a
 * captured graph stays valid) across sfa_batch_update calls.
 */
int sfa_batch_reserve(int32_t max_texts, uint64_t max_tiles, uint32_t nr_max, const sfa_launch_opts *opts,
                      sfa_batch_t *out);

/*
 * sfa_batch_update -- replaces the work list of a reserved plan by k texts
 * (same arguments as sfa_batch_create).  Builds it on the host in pinned
 * staging and enqueues its upload on `stream`; allocates nothing for SFA-mode
 * handles (simulation-mode texts may grow their handle's scratch).  Issue the
 * update and the following launch on the same stream.  INVALID when the texts
 * exceed the plan's capacity or an automaton has more than nr_max states.
 */
int sfa_batch_update(sfa_batch_t b, const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens,
                     int32_t k, sfa_stream_t stream);

/*
 * sfa_batch_update_host -- sfa_batch_update for texts still on the host: the
 * lens[i] bytes at h_texts[i] are copied to d_dst[i] (device, the caller's
 * buffer) on `stream`, then the work list is replaced by the k texts at
 * d_dst (as sfa_batch_update).  Texts in host memory that the device can
 * read (pinned memory mapped into its address space, as cudaHostAlloc and
 * torch's pin_memory give; checked with cudaPointerGetAttributes) are copied
 * by one kernel for the whole batch, at the host link's bandwidth, fastest
 * when d_dst[i] and h_texts[i] have the same address modulo 16; other texts
 * take one cudaMemcpyAsync each (synchronous for pageable memory).  The
 * serving loop's copy-in; the paper has no counterpart.  Errors as
 * sfa_batch_update, plus CUDA when a copy cannot be enqueued (copies
 * enqueued before the failure stay enqueued).
 */
int sfa_batch_update_host(sfa_batch_t b, const sfa_handle_t *hs, const uint8_t *const *h_texts,
                          uint8_t *const *d_dst, const uint64_t *lens, int32_t k, sfa_stream_t stream);

/* sfa_batch_launch -- enqueue the planned work; d_out: device, k results in
 * the order of the texts given to sfa_batch_create.  Launches of one plan
 * must not overlap on the GPU. */
int sfa_batch_launch(sfa_batch_t b, sfa_result *d_out, sfa_stream_t stream);

/* sfa_batch_graph_launch -- as sfa_batch_launch, but through a CUDA graph
 * captured on the first call for this (d_out) and replayed afterwards. */
int sfa_batch_graph_launch(sfa_batch_t b, sfa_result *d_out, sfa_stream_t stream);

/* sfa_batch_destroy -- frees a plan (NULL is fine); no launch may be in flight. */
void sfa_batch_destroy(sfa_batch_t b);

/* sfa_match_batch -- create + launch + destroy (destroy after the stream
 * synchronises).  For repeated batches keep a plan instead. */
int sfa_match_batch(const sfa_handle_t *hs, const uint8_t *const *d_texts, const uint64_t *lens,
                    int32_t k, sfa_result *d_out, sfa_stream_t stream);

/* ---- serving ------------------------------------------------------------- */
/*
 * A continuous-batching match server over resident automata (the paper has
 * no counterpart: it is the serving loop around sfa_batch_*).  Requests are
 * queued by sfa_server_submit; each sfa_server_progress call completes the
 * batches the device has finished and admits queued requests, first in,
 * first out, into free batch slots while the device text arena has room:
 * their texts are copied into the arena (one cudaMemcpyAsync each) and
 * matched by one persistent launch per batch on the slot's stream.  No call
 * waits for the device, and nothing is allocated after sfa_server_create.
 * Every result equals the text's result alone (sfa_match).  One thread at a
 * time may call a server's functions.
 */
typedef struct sfa_server *sfa_server_t;

typedef struct {
    uint64_t hbm_budget;      /* device bytes of the text arena (0 = 4 GiB) */
    int32_t max_batch;        /* requests per launch (0 = 256) */
    int32_t slots;            /* batches in flight, one stream each (0 = 3) */
    uint32_t chunk_bytes;     /* chunk length of the batch plans (0 = 1024) */
    uint32_t block_threads;   /* CTA size of the batch plans (0 = 512) */
    uint32_t flags;           /* SFA_SERVER_* */
    uint32_t reserved;
} sfa_server_opts;

#define SFA_SERVER_TIMING 1u  /* record device timestamps of every batch (sfa_server_spans) */

/* The device timeline of one batch (SFA_SERVER_TIMING): CUDA-event times in
 * ms since sfa_server_create, recorded on the batch's slot stream before the
 * copy-in, between the copy-in and the match, and after the match.  An event
 * is stamped when its stream reaches it, so a span also covers the time the
 * batch's work waited for the device behind other slots' work. */
typedef struct {
    int32_t slot;             /* the batch slot (one stream each) */
    int32_t requests;         /* requests in the batch */
    uint64_t bytes;           /* text bytes of the batch */
    float copy_start_ms;
    float copy_end_ms;        /* = start of the match */
    float match_end_ms;
    float reserved;
} sfa_batch_span;

/* sfa_server_spans -- the spans of finished batches not returned yet, up to
 * cap of them in out[] (*n of them), oldest first; 0 spans without
 * SFA_SERVER_TIMING. */
int sfa_server_spans(sfa_server_t s, sfa_batch_span *out, int32_t cap, int32_t *n);

typedef struct {
    uint64_t tag;             /* the caller's tag of the request */
    sfa_result result;
} sfa_completion;

typedef struct {
    uint64_t queued;              /* submitted, not yet admitted */
    uint64_t in_flight;           /* admitted, batch not yet finished */
    uint64_t completed_waiting;   /* finished, not yet returned */
    uint64_t batches;             /* launches so far */
    uint64_t requests;            /* requests admitted so far */
    uint64_t arena_used;          /* arena bytes held by admitted requests */
} sfa_server_stats_t;

/* sfa_server_create -- n automata (handles on the current device; the
 * handles must outlive the server); opts NULL = defaults.  Allocates the
 * arena, the batch plans, streams, events and pinned result buffers
 * (synchronous).  Errors: INVALID, HOST_ONLY, NO_DEVICE, OOM, CUDA, and
 * UNSUPPORTED for a handle with 16-bit state ids (sfa_info id_bits = 16). */
int sfa_server_create(const sfa_handle_t *automata, int32_t n, const sfa_server_opts *opts, sfa_server_t *out);

/* sfa_server_submit -- queue one request: automaton index in [0, n), host
 * text of len bytes (pinned for asynchronous copies; it must stay valid and
 * unmodified until the request completes), and a tag returned with its
 * result.  INVALID for a bad index, a NULL text with len > 0, or a text
 * longer than the arena less 15 bytes (a text is placed at its host
 * address's offset modulo 16 in its arena range). */
int sfa_server_submit(sfa_server_t s, int32_t automaton, const uint8_t *h_text, uint64_t len, uint64_t tag);

/* sfa_server_submit_many -- k requests at once (arrays of automaton indices,
 * host texts, lengths and tags, as for sfa_server_submit); all are queued,
 * in order, or none (INVALID). */
int sfa_server_submit_many(sfa_server_t s, int32_t k, const int32_t *automata, const uint8_t *const *h_texts,
                           const uint64_t *lens, const uint64_t *tags);

/* sfa_server_progress -- complete finished batches, admit and launch queued
 * requests, and return up to cap completions in done[] (*n_done of them;
 * the rest are kept for later calls).  A failure to enqueue a batch returns
 * its error and leaves those requests at the head of the queue. */
int sfa_server_progress(sfa_server_t s, sfa_completion *done, int32_t cap, int32_t *n_done);

/* sfa_server_stats -- counters of the server's queue, slots and arena. */
int sfa_server_stats(sfa_server_t s, sfa_server_stats_t *out);

/* sfa_server_destroy -- waits for the slots' streams, then frees everything
 * (NULL is fine).  Requests not yet completed are dropped. */
void sfa_server_destroy(sfa_server_t s);

/* The server's arena allocator, on its own (host only; offsets, no memory):
 * first fit, ranges rounded up to 256 bytes, free neighbours merged.
 * sfa_arena_alloc returns OOM when no free range is long enough;
 * sfa_arena_release returns INVALID for a range that is not held. */
typedef struct sfa_arena *sfa_arena_t;
sfa_arena_t sfa_arena_create(uint64_t size);
int sfa_arena_alloc(sfa_arena_t a, uint64_t n, uint64_t *off);
int sfa_arena_release(sfa_arena_t a, uint64_t off, uint64_t n);
uint64_t sfa_arena_used(sfa_arena_t a);
void sfa_arena_destroy(sfa_arena_t a);

/* ---- regular expressions (the front end of Sect. VI) --------------------- */
/*
 * The pipeline of the paper's matcher (Sect. VI): a regular expression to
 * an NFA by McNaughton and Yamada's position construction, to a DFA by the
 * subset construction (Alg. 1), minimised (partition refinement), then the
 * D-SFA by sfa_compile.  Host only.  Syntax (bytes): literals; escapes \n \t
 * \r \f \v \0 \xHH and \ before a non-alphanumeric byte; \d \D \w \W \s \S;
 * '.' (every byte but newline, every byte with SFA_REGEX_DOTALL); classes
 * [...] with ranges and [^...]; groups (...) and (?:...); |; * + ? {m} {m,}
 * {m,n} (m, n <= 1000).  No anchors, back-references or lazy quantifiers.
 * The language is matched against whole prefixes of a text (a position is
 * counted when the prefix ending there is in the language); with
 * SFA_REGEX_SEARCH the automaton is that of (any byte)* r, so a position is
 * counted when an occurrence of r ends there.
 */
#define SFA_REGEX_SEARCH      1u
#define SFA_REGEX_DOTALL      2u
#define SFA_REGEX_NO_MINIMIZE 4u   /* keep the subset automaton as built */

typedef struct {
    int32_t nq;               /* DFA states (the empty set of NFA states, a dead
                                 state, included when reachable) */
    int32_t q0;               /* initial state (0) */
    int32_t positions;        /* positions of the expression (NFA states - 1) */
    int32_t subset_states;    /* states of the subset construction, before minimising */
    int32_t ncls;             /* byte classes of the expression */
    int32_t reserved;
} sfa_regex_info;

/*
 * sfa_regex_dfa -- the (minimal) DFA of a regular expression.
 *   pattern, len  the expression's bytes (no terminator needed)
 *   cap           capacity of delta/accept in states
 *   delta         host int32[cap * 256] or NULL: written row-major as for
 *                 sfa_compile, states numbered breadth first from q0 = 0
 *   accept        host uint8[cap] or NULL (both or neither)
 *   info          host, optional: sizes (filled also when the DFA does not fit)
 *   err_pos       host, optional: byte offset of a syntax error
 * Errors: INVALID (syntax, with *err_pos), UNSUPPORTED (more than cap states,
 * or 4096 positions after {m,n} are expanded), OOM.
 */
int sfa_regex_dfa(const char *pattern, size_t len, uint32_t flags, int32_t cap, int32_t *delta, uint8_t *accept,
                  sfa_regex_info *info, size_t *err_pos);

/* sfa_regex_compile -- sfa_regex_dfa then sfa_compile (up to 4095 DFA states). */
int sfa_regex_compile(const char *pattern, size_t len, uint32_t flags, const sfa_compile_opts *opts,
                      sfa_handle_t *out);

/*
 * sfa_regex_nsfa_states -- the size of the N-SFA of the expression's
 * position NFA (Definition 1 over correspondences, built by Alg. 4: f_I(q) =
 * {q}, f_next(q) = the union of delta(q', sigma) over q' in f(q)); Theorem 2
 * bounds it by 2^(n^2) for n NFA states.  The matcher runs D-SFAs; this
 * reports what the nondeterministic construction would cost.  UNSUPPORTED
 * (with *n_states = cap) past cap states.
 */
int sfa_regex_nsfa_states(const char *pattern, size_t len, uint32_t flags, uint64_t cap, uint64_t *n_states);

/* ---- launch statistics (for benchmarks) --------------------------------- */
/* Number of kernels the library enqueued since load (all entry points). */
uint64_t sfa_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* SFA_H */
