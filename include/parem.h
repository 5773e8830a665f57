/*
 * parem.h -- C ABI of libparem: chunked speculative DFA matching on one GB300 (sm_103a).
 *
 * The library implements the data-parallel hot path of PaREM (Memeti & Pllana,
 * "PaREM: A Novel Approach for Parallel Regular Expression Matching", CSE 2014):
 * the text is cut into chunks, every chunk is run from the speculated candidate set of
 * initial states (the states reachable on the last symbol of the preceding chunk), the
 * per-chunk state maps are composed in text order to find each chunk's true start, and
 * the matches are counted and emitted (Section II-B, Algorithm 1).  The result is exactly
 * that of the plain sequential DFA run of Section II-A.
 *
 * Conventions shared by every entry point
 *   - Every call returns an int status: PAREM_OK (0) or a negative PAREM_ERR_* code.
 *     parem_strerror() gives a message.  Nothing is written to the caller's outputs when
 *     a call fails before launching GPU work (INVALID_ARG, OOM).
 *   - Host pointers are read during the call only; the library copies what it keeps.
 *   - "device pointer" means memory of the current CUDA device (cudaMalloc'd, or a
 *     PyTorch CUDA tensor).  The caller owns text and position buffers.
 *   - Work is ordered on the CUDA stream passed as `void* stream` (a cudaStream_t; NULL is
 *     the legacy default stream).  Calls are synchronous with respect to `*out`: when they
 *     return, the result is on the host and the positions are written.
 *   - Calls on distinct streams may run concurrently from different host threads; the
 *     library keeps its scratch memory per (device, stream).
 *   - State numbers in and out are the caller's original numbers; PAREM_NONE stands for
 *     the dead state (the run has met an undefined transition or a byte outside the
 *     alphabet).
 *
 * Semantics (readings of the paper, the same as the CPU oracle's)
 *   - A transition entry PAREM_NONE is undefined ("Tt[q][c] in Q" fails in Algorithm 1);
 *     a byte whose symbol is PAREM_NONE16 is outside the alphabet.  Both lead to an
 *     absorbing, non-accepting dead state.
 *   - A match is counted after each symbol whose transition lands in F (Algorithm 1's
 *     found++), at the 0-based index of that symbol; the start state is never counted.
 *     Positions are ascending, one per index.
 *   - accepted = (final state in F) (Section II-A); for an empty text it is (q0 in F).
 */
#ifndef PAREM_H
#define PAREM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PAREM_NONE 0xFFFFFFFFu   /* undefined transition / dead state */
#define PAREM_NONE16 0xFFFFu     /* byte outside the alphabet */

#define PAREM_OK 0
#define PAREM_ERR_INVALID_ARG (-1) /* null pointer, out-of-range entry or size */
#define PAREM_ERR_OOM (-2)         /* device or host allocation failed */
#define PAREM_ERR_CAPACITY (-3)    /* more matches than `capacity`; count is still exact */
#define PAREM_ERR_TIMEOUT (-4)     /* a bounded device-side wait ran out */
#define PAREM_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define PAREM_ERR_INTERNAL (-6)    /* a device-side self-check failed */
#define PAREM_ERR_UNSUPPORTED (-7) /* valid request outside what the library supports */
#define PAREM_ERR_TOO_LARGE (-8)   /* parem_match_noalloc: the request needs more scratch than
                                      its fixed area (PAREM_NOALLOC_SCRATCH_BYTES) holds */

/* Size of the fixed device scratch area used by parem_match_noalloc (16 MiB). */
#define PAREM_NOALLOC_SCRATCH_BYTES (16u << 20)

typedef struct parem_dfa parem_dfa; /* opaque; tables resident on one device */

typedef struct {
  uint32_t final_state; /* state after the last symbol (original numbering), or PAREM_NONE */
  uint8_t accepted;     /* final_state in F */
  uint8_t reserved[3];
  uint64_t match_count; /* number of match positions in the whole text (exact) */
  uint64_t n_written;   /* positions written: min(match_count, capacity), 0 if none asked */
} parem_result;

/* Description of a prepared DFA (host-side planning data). */
typedef struct {
  uint32_t n_states;        /* states as given */
  uint32_t n_symbols;       /* symbols as given */
  uint32_t compact_states;  /* states on the device, including the dead state if any */
  uint32_t n_classes;       /* distinct transition columns among the symbols the bytes use */
  uint32_t has_dead;        /* 1 when a dead state was added */
  uint32_t entry_bytes;     /* 1 (<= 256 compact states) or 2 */
  uint32_t layout;          /* 0: byte-indexed table in shared memory, 1: class-indexed table
                               in shared memory, 2: class-indexed table in global memory (L2);
                               3 and 4: as 1 and 2 with 2-byte column offsets;
                               6: as 0, plus a table that advances 4 bytes per lookup in the
                               main run (small DFAs whose bytes 0..K-2 are distinct classes
                               and whose other bytes share one class);
                               7: class table in shared memory whose column is computed from
                               the byte (all bytes outside one ASCII window of at most 64
                               values and one extra byte share a class) */
  uint32_t table_bytes;     /* bytes of the device transition table */
  uint32_t max_candidates;  /* largest candidate set |img(c) \ {dead}| over classes */
  uint32_t sync_estimate;   /* symbols after which a candidate set has shrunk to one state on
                               random input (median of seeded trials; 0 when no set has two
                               states; 0xFFFFFFFF when a trial did not synchronise) */
  double mean_candidates;   /* mean candidate set size over the 256 byte values */
  uint32_t pair_hot_states; /* > 0 once the two-byte stride variant (layout 8) has been learned
                               from a text: its hot states; scans use it from then on */
  uint32_t reserved;
} parem_dfa_info;

/* Options of parem_match_ex; zero-initialise, then set what you need. */
typedef struct {
  uint32_t start_state;     /* with use_start_state = 1: the state carried in from the end of
                               a previous piece of a stream (original numbering), so a long
                               text can be matched piecewise; positions are then relative to
                               this piece.  Ignored otherwise (the run starts at q0). */
  uint32_t enumerate_all;   /* 1: speculate every state as a chunk's candidate (the general
                               enumeration approach the paper compares against, Section IV-A)
                               instead of the candidate set of Algorithm 1. */
  uint64_t segment_bytes;   /* bytes per lane segment; 0 = planner's choice.  Rounded up to
                               a multiple of 128. */
  uint32_t warps_per_block; /* 0 = planner's choice (1..32) */
  uint32_t spec_cap_bytes;  /* longest speculative prefix before a segment is treated as not
                               converging; 0 = planner's choice */
  uint64_t wait_budget_cycles; /* bound of every device-side wait, in SM clock cycles;
                                  0 = about 2 seconds */
  int64_t debug_skip_publish_chunk; /* test hook, 0 = off: a positive k makes chunk k never
                                       publish its state, so its successor's bounded wait runs
                                       out and the call returns PAREM_ERR_TIMEOUT */
  uint32_t record_kernel_times; /* 1: record CUDA events around each kernel of the call on the
                                   call's stream; read them with parem_last_stats */
  uint32_t use_start_state; /* 1: start from start_state instead of q0 */
  uint32_t pair_mode;       /* the two-byte stride variant of a DFA with computed columns (layout
                               7): PAREM_PAIR_AUTO (0) learns its hot states from the first scan
                               of at least 64 MiB and uses it from the next scan on;
                               PAREM_PAIR_LEARN (1) learns from this call's text (at least 4 KiB)
                               if not learned yet; PAREM_PAIR_OFF (2) neither learns nor uses it
                               in this call.  Results are the same in every mode. */
} parem_match_opts;

#define PAREM_PAIR_AUTO 0u
#define PAREM_PAIR_LEARN 1u
#define PAREM_PAIR_OFF 2u

/* What the last scan on a (device, stream) did: its plan and, when record_kernel_times was
 * set, the device time of each kernel. */
typedef struct {
  float scan_ms;            /* pass 1: speculation, main run and look-back (-1 if not timed) */
  float emit_ms;            /* pass 2: position emission (0 if not launched, -1 if not timed) */
  uint64_t segment_bytes;   /* S: bytes per lane segment */
  uint64_t rows;            /* full segments */
  uint64_t chunks;          /* 32-segment chunks (look-back units) */
  uint32_t blocks;          /* persistent thread blocks of pass 1 */
  uint32_t warps_per_block;
  uint32_t candidate_regs;  /* candidate registers per lane in the speculation (1 or 8) */
  uint32_t spec_cap_bytes;  /* longest speculative prefix per segment */
  uint32_t kernels;         /* kernels launched by the call */
  uint32_t emit_replays;    /* rows whose positions the emit pass replayed (not recorded in pass 1) */
  uint32_t emit_max_window; /* longest window (bytes) the emit pass replayed */
  uint32_t nonconv_rows;    /* rows whose candidates did not merge within the speculation cap
                               (resolved through slot maps or a run from the resolved start) */
  uint32_t conv_max;        /* longest speculative prefix a row needed before its candidates
                               merged (bytes); later plans for the DFA use longer rows */
  /* SM cycles of the warps owning chunks, summed over chunks: speculation (including slot
     maps), main run, resolution (waits on predecessors, look-back, row records) */
  uint64_t cycles_spec, cycles_main, cycles_resolve;
  uint64_t cycles_bitmap, cycles_lane;  /* parts of cycles_spec: the bitmap phase of large
                                           candidate sets, the lane phase of the survivors */
  /* Speculation work (the overhead of Algorithm 1's candidate runs over one run per byte):
     table lookups by candidate runs before they merged, summed over rows -- counted as the
     live candidates after each merge check times the steps to the next check, so an upper
     bound within one check interval (4 or 16 steps) -- plus every candidate's run of a row
     resolved through a slot map.  Divide by the text bytes for lookups per byte. */
  uint64_t spec_lookups;
  uint32_t layout;          /* table layout of the scan (8: the two-byte stride variant) */
  uint32_t pair_hot_states; /* hot states of the two-byte stride table (layout 8), else 0 */
} parem_stats;

/*
 * parem_load_dfa -- prepare a DFA (Q, Sigma, delta, q0, F) (Section II-A) and upload it
 * to the current device.  This is the "transition table Tt, set of final states F" input
 * of Algorithm 1; the table plays the role of the adjacency matrix that the paper's
 * graph-based code generator emits (Section III).
 *   table          host, n_states * n_symbols uint32, row-major table[q * n_symbols + a];
 *                  each entry < n_states or PAREM_NONE.
 *   n_states       1 .. 65535.
 *   n_symbols      1 .. 256.
 *   byte_to_symbol host, 256 uint16: the symbol of each text byte (< n_symbols) or
 *                  PAREM_NONE16; NULL = identity (byte b is symbol b when b < n_symbols).
 *   start          q0 < n_states.
 *   accept         host, n_states uint8 flags (nonzero = in F).
 *   out            receives the handle; free it with parem_free_dfa.
 * Errors: INVALID_ARG, OOM, CUDA.  Host preparation: dead-state completion, merging of
 * identical symbol columns into classes, renumbering (accepting states last), the
 * candidate lists img(c) and the slot table rank(c, q) used by the speculation.
 */
int parem_load_dfa(const uint32_t* table, uint32_t n_states, uint32_t n_symbols,
                   const uint16_t* byte_to_symbol, uint32_t start, const uint8_t* accept,
                   parem_dfa** out);

/*
 * Regular expressions (host only, no GPU): the operators of the paper's Table III --
 * concatenation ab, Kleene star a*, union a|b, positive closure a+, range [0..9] (also
 * written [0-9]; [^..] negates a set), optionality a?, group ( ) -- compiled by the
 * McNaughton-Yamada-Thompson construction and the subset construction (Section III) into a
 * DFA for parem_load_dfa, which is then minimized.  A byte stands for itself, '\' escapes the next one (\n \t \r
 * \0 \xHH), '.' is any byte, and an empty alternative matches the empty string.  Bytes
 * that every edge treats alike share one symbol, so the table has one column per class.
 *
 * flags: 0 = search: the DFA is in an accepting state after position j exactly when some
 * suffix of text[0..j], possibly empty, matches (the DFA of Sigma* R), so parem_match counts
 * and emits every such j; PAREM_REGEX_ANCHORED: when text[0..j] matches.
 * max_states caps the DFA (0: 65,535).  The DFA state 0 is the start; table entries are
 * PAREM_NONE where no match can continue.
 * Errors: INVALID_ARG (null pointer, unknown flag, syntax error), TOO_LARGE (more states
 * than max_states, or a pattern longer than 16 KiB), OOM.
 */
#define PAREM_REGEX_ANCHORED 1u
typedef struct parem_regex parem_regex;
int parem_regex_compile(const char* pattern, uint64_t len, uint32_t flags, uint32_t max_states,
                        parem_regex** out);
/* The DFA's size: states and symbols (byte classes). */
int parem_regex_info(const parem_regex* re, uint32_t* n_states, uint32_t* n_symbols);
/* The DFA in parem_load_dfa's form: table (n_states * n_symbols, row-major), the 256-entry
 * byte-to-symbol map, accept flags (n_states) and the start state; caller-owned buffers. */
int parem_regex_export(const parem_regex* re, uint32_t* table, uint16_t* byte_to_symbol, uint8_t* accept,
                       uint32_t* start);
/* parem_load_dfa of the compiled DFA. */
int parem_regex_load(const parem_regex* re, parem_dfa** out);
void parem_regex_free(parem_regex* re);

/* Host-only preparation of the same inputs, without touching the GPU: validates them and
 * fills *info.  Errors: INVALID_ARG. */
int parem_prepare_info(const uint32_t* table, uint32_t n_states, uint32_t n_symbols,
                       const uint16_t* byte_to_symbol, uint32_t start, const uint8_t* accept,
                       parem_dfa_info* info);

/* Information about a loaded DFA.  Errors: INVALID_ARG. */
int parem_dfa_get_info(const parem_dfa* dfa, parem_dfa_info* info);

/* Free a DFA (NULL is ignored).  Synchronises the device first. */
void parem_free_dfa(parem_dfa* dfa);

/*
 * parem_match -- run the DFA over a device-resident text (Algorithm 1: chunking,
 * candidate speculation R = S n L, candidate runs, join; Section II-B).
 *   dfa        from parem_load_dfa (the same device must be current).
 *   text       device pointer, any alignment; may be NULL when len == 0.
 *   len        bytes; at most 2^45.
 *   positions  device pointer to `capacity` uint64 slots, or NULL to count only.  Receives
 *              the first min(match_count, capacity) match positions, ascending.
 *   stream     cudaStream_t or NULL.
 *   out        host; receives final state, accepted, match_count, n_written.
 * Errors: INVALID_ARG, OOM, CUDA, TIMEOUT, INTERNAL; CAPACITY when positions != NULL and
 * match_count > capacity (out is still filled, and exact).
 */
int parem_match(const parem_dfa* dfa, const uint8_t* text, uint64_t len, uint64_t* positions,
                uint64_t capacity, void* stream, parem_result* out);

/* parem_match with options (carry-in start state, enumeration mode, tuning, test hook).
 * opts may be NULL (same as parem_match).  Errors as parem_match. */
int parem_match_ex(const parem_dfa* dfa, const uint8_t* text, uint64_t len, uint64_t* positions,
                   uint64_t capacity, const parem_match_opts* opts, void* stream, parem_result* out);

/*
 * parem_match_host -- the same scan for a text in HOST memory: the library copies the text
 * to the device in pieces (overlapping the copies with the scan of earlier pieces, each
 * piece started from the state the previous one ended in) and copies the positions back.
 *   text       host pointer (pinned memory is fastest; pageable works).
 *   positions  host pointer to `capacity` uint64, or NULL to count only.
 * Errors as parem_match.
 */
int parem_match_host(const parem_dfa* dfa, const uint8_t* text, uint64_t len, uint64_t* positions,
                     uint64_t capacity, void* stream, parem_result* out);

/*
 * parem_match_noalloc -- parem_match for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this entry point exists for users of the library.  Some
 * callers must not have a library call cudaMalloc behind their back: applications whose
 * device memory is handed to their own pool allocator at start-up (so a library allocation
 * fails, or fragments the pool they manage), and latency-sensitive code that cannot afford
 * the implicit device-wide synchronisation that allocating and freeing device memory may
 * cause.  parem_match keeps per-stream scratch that it allocates on first use and grows on
 * demand; this variant runs the same kernels with all of their scratch (ticket counter,
 * result word, chunk status words, per-row records and slot maps) in one fixed array of
 * PAREM_NOALLOC_SCRATCH_BYTES in device memory, defined statically in the library.  It calls
 * no cudaMalloc, cudaFree or other allocating routine.
 *   Arguments, results and errors are those of parem_match, plus PAREM_ERR_TOO_LARGE when
 *   the scan of this text would need more scratch than the fixed area holds: 8 bytes per
 *   32-row chunk, 112 bytes per row when positions are requested, and, for DFAs whose
 *   unmerged rows go through slot maps (at most 32 candidates, or no synchronisation), 8
 *   bytes per candidate per row.  With the default plan a 16 MiB area holds hundreds of MiB
 *   of text for the count, and about 100-150 MiB when positions are requested.
 *   Nothing is written to the outputs in that case.
 *   Plans are those of parem_match for the same DFA: both entry points learn from every scan
 *   (how long the DFA's candidates take to merge, how dense its matches are), so a DFA whose
 *   earlier scans found dense matches gets the streaming emit pass here as well.
 *   Every GPU that loads the library holds the array until the process exits.  The first
 *   call on a device looks up the array's device address (cudaGetSymbolAddress, with that
 *   device current); make that first call before any stream capture begins.  All calls share
 *   the one array: the library clears the parts that must start at zero on every call, but
 *   calls whose work overlaps on the GPU (different streams, or host threads) race on it and
 *   give wrong results; serialise them.
 */
int parem_match_noalloc(const parem_dfa* dfa, const uint8_t* text, uint64_t len, uint64_t* positions,
                        uint64_t capacity, void* stream, parem_result* out);

/*
 * parem_pair_preview -- host-only look at the two-byte stride variant (table layout 8) that
 * scans learn for a DFA with computed columns (layout 7); needs no GPU.
 *
 * The paper's candidate runs take one table lookup per symbol.  For texts of lowercase
 * letters and spaces the library also keeps, for the H states a run visits most (the hot
 * states, learned from a sample of the first large text), a table of the state reached after
 * two bytes: byte codes f = b & 0x1F (0 for the space 0x20, 1..26 for a..z), pair index
 * 27 f0 + f1, entry = hot index of the state after both bytes, or H ("escape") when the
 * state after either byte is accepting or the state after both is not hot.  Row H is all H.
 * The main run takes a 16-byte vector two bytes per lookup when it starts in a hot state,
 * holds only such bytes and never escapes; otherwise it runs the vector byte by byte.
 * This call plans the variant from `sample` exactly as a scan would and reports it:
 *   sample       host text, sample_len bytes (one window; the first 64 bytes only settle).
 *   info         receives the base layout, H, whether the variant pays (a scan would keep it)
 *                and the estimated share of 32-lane vector steps needing the byte loop.
 *   hot_states   optional, H uint32: original id of hot state e (the row order).
 *   pair_table   optional, (H + 1) * 729 bytes (info->pair_table_bytes): the rows.
 * Errors: INVALID_ARG (as parem_load_dfa), CAPACITY (pair_table_cap too small).
 */
typedef struct {
  uint32_t layout;            /* layout the DFA prepares to (the variant needs 7) */
  uint32_t hot_states;        /* H, 0 when no variant can be planned */
  uint32_t accepted;          /* 1: a scan would use the variant */
  uint32_t reserved;
  double warp_slow_share;     /* estimated share of 32-lane vector steps needing the byte loop */
  uint64_t pair_table_bytes;  /* (H + 1) * 729 */
} parem_pair_info;

int parem_pair_preview(const uint32_t* table, uint32_t n_states, uint32_t n_symbols,
                       const uint16_t* byte_to_symbol, uint32_t start, const uint8_t* accept,
                       const uint8_t* sample, uint64_t sample_len, parem_pair_info* info,
                       uint32_t* hot_states, uint8_t* pair_table, uint64_t pair_table_cap);

/*
 * Batched matching: many (text, DFA) pairs in one persistent launch.
 *
 * The batch is planned once (parem_batch_create) and run any number of times
 * (parem_batch_run), e.g. after the caller refills the same text buffers.  Planning assigns
 * each item its rows of S bytes, lays out every item's scratch in one allocation, writes the
 * per-item descriptors (scan parameters and TMA tensor maps) to device memory, and captures
 * the work (clearing the scratch, the persistent scan kernel, the emit kernel, the copy of
 * the results to pinned host memory) into one CUDA graph.  In the persistent kernel each
 * thread block serves one DFA at a time, with that DFA's table staged in shared memory (or
 * read from L2 when it is too large), and moves to another DFA when the first runs out of
 * chunks.  Every item's result is exactly that of parem_match on it (Algorithm 1 per item).
 */
typedef struct parem_batch parem_batch;

typedef struct {
  const parem_dfa* dfa;   /* loaded on the current device */
  const uint8_t* text;    /* device pointer, any alignment (NULL when len == 0) */
  uint64_t len;
  uint64_t* positions;    /* device pointer or NULL (count only) */
  uint64_t capacity;      /* slots in positions */
} parem_batch_item;

/* Speculation form of a batch DFA (Algorithm 1's speculation step over the candidate set of
 * each row; the forms differ only in how a warp holds and merges the candidates):
 *   GROUPED      a few lanes per row hold its candidates, 32/G rows at once (sets of <= 32)
 *   WARP         one row at a time, candidates over 32 lanes x 8 registers, merged by
 *                warp votes on equal states (sets of <= 256)
 *   WARP_BITMAP  one row at a time, merged through a bitmap of the states in shared memory
 *                (any set size; DFAs of at most 16,384 states)
 * AUTO (0) picks by the candidate-set size and the DFA's estimated synchronisation length. */
#define PAREM_BATCH_SPEC_AUTO 0u
#define PAREM_BATCH_SPEC_GROUPED 1u
#define PAREM_BATCH_SPEC_WARP 2u
#define PAREM_BATCH_SPEC_WARP_BITMAP 3u

typedef struct {
  uint32_t autotune;        /* 1: choose each DFA's segment size and speculation form by timing
                               candidates on its own items, and the block shape by timing the
                               whole batch (several trial runs during parem_batch_create) */
  uint32_t warps_per_block; /* 0 = 24, or with autotune the faster of 24 and 16; 1..16 = 16 warps
                               (128 registers each); > 16 = 24 (80 registers each) */
  uint64_t segment_bytes;   /* 0 = planner/autotuner; else the same S for every item */
  uint32_t use_graph;       /* 0: launch the kernels directly in parem_batch_run; else (default
                               when the struct is NULL) replay the captured CUDA graph */
  uint32_t spec;            /* PAREM_BATCH_SPEC_*: the form for every DFA where it applies
                               (others keep AUTO's); not AUTO also stops the autotuner trying
                               forms */
} parem_batch_opts;

/* The configuration a batch chose for one item (planner or autotuner). */
typedef struct {
  uint64_t segment_bytes;   /* S (0: the text is shorter than one row) */
  uint32_t spec;            /* PAREM_BATCH_SPEC_GROUPED, _WARP or _WARP_BITMAP */
  uint32_t warps_per_block; /* of the whole batch's launch: 16 or 24 */
  uint32_t smem_table;      /* 1: the DFA's table is staged in shared memory, 0: read from L2 */
  uint32_t reserved;
} parem_batch_config;

/* Plan a batch of n_items items (host array, copied) on the current device.  Errors:
 * INVALID_ARG, OOM, CUDA. */
int parem_batch_create(const parem_batch_item* items, uint32_t n_items, const parem_batch_opts* opts,
                       parem_batch** out);

/* Run the batch on `stream` and wait for it.  Errors: CUDA, TIMEOUT, INTERNAL; CAPACITY when some
 * item had more matches than its capacity (its result is still exact). */
int parem_batch_run(parem_batch* batch, void* stream);

/* Results of the last run, in the order of the items given to parem_batch_create. */
int parem_batch_results(const parem_batch* batch, parem_result* out);

/* Segment size chosen for item i (planner or autotuner).  Errors: INVALID_ARG. */
int parem_batch_item_segment(const parem_batch* batch, uint32_t i, uint64_t* segment_bytes);

/* Everything chosen for item i (given order): segment size, speculation form, block shape,
 * table tier.  Errors: INVALID_ARG. */
int parem_batch_item_config(const parem_batch* batch, uint32_t i, parem_batch_config* out);

/* Counters of the last run summed over the batch's items (the plan fields are 0; unmerged
 * rows, longest merge, kernels and the cycle counters are filled).  Errors: INVALID_ARG. */
int parem_batch_stats(const parem_batch* batch, parem_stats* out);

/* Free a batch (NULL is ignored). */
void parem_batch_free(parem_batch* batch);

/*
 * Request server: continuous batching of independent match requests.
 *
 * Algorithm 1 applies to each request on its own (every response equals parem_match on that
 * request); the server only decides which requests share a launch.  A dispatcher thread
 * takes the waiting requests in arrival order, as many as fit one batch (a request-count and
 * a text-byte limit, and the scratch and descriptor space of a pre-allocated arena: memory
 * admission), plans them into the arena and launches the batch kernels on that arena's
 * stream.  With two or more arenas the next batch is launched while the previous one runs,
 * so requests that arrive meanwhile start as soon as thread blocks of the running batch
 * retire.  A completion thread answers the batches as they finish, in any order (a batch
 * holding a long request does not hold back later batches), and queues their responses;
 * a request without a positions buffer is answered as soon as the kernel has its result,
 * before the rest of its batch is done.  Nothing is allocated per request or per batch.  Mode PAREM_SERVE_FIFO instead
 * runs the requests one at a time through parem_match, in arrival order (the plain
 * comparison).
 *
 * Texts and position buffers are device memory owned by the caller; they must stay valid
 * until the request's response has been polled.  Timestamps are nanoseconds of the steady
 * clock that parem_clock_ns reads.
 */
typedef struct parem_server parem_server;

#define PAREM_SERVE_BATCH 0u
#define PAREM_SERVE_FIFO 1u

typedef struct {
  uint32_t mode;                 /* PAREM_SERVE_BATCH (default) or PAREM_SERVE_FIFO */
  uint32_t arenas;               /* batches in flight (0 = 256): a batch that holds a long request
                                    keeps its arena until that request is done, so many
                                    arenas keep the GPU busy behind it */
  uint32_t max_items;            /* requests per batch (0 = 4096) */
  uint32_t reserved0;
  uint64_t max_batch_bytes;      /* text bytes per batch (0 = 1 GiB) */
  uint64_t arena_scratch_bytes;  /* device scratch per arena (0 = 128 MiB) */
  uint64_t reserved[4];
} parem_server_opts;

typedef struct {
  uint32_t dfa_index;        /* index into the DFAs given to parem_server_create */
  uint32_t reserved0;
  const uint8_t* text;       /* device */
  uint64_t len;
  uint64_t* positions;       /* device, or NULL for the count only */
  uint64_t capacity;
  uint64_t tag;              /* returned in the response */
  int64_t arrival_ns;        /* arrival time (steady clock); 0 = the time of submission */
} parem_request;

typedef struct {
  uint64_t tag;
  int32_t status;            /* as parem_match: OK, CAPACITY, TIMEOUT, INTERNAL, TOO_LARGE (the
                                request alone exceeds an arena), INVALID_ARG */
  uint32_t batch_size;       /* requests in the launch that served this one */
  parem_result result;
  int64_t arrival_ns;
  int64_t launch_ns;         /* when its batch was launched */
  int64_t done_ns;           /* when its result was on the host */
} parem_response;

typedef struct {
  uint64_t submitted, answered, batches, bytes;
  uint64_t max_batch;        /* largest batch launched */
  uint64_t kernels;          /* kernel launches so far */
  uint64_t reserved[2];
} parem_server_stats;

/* Create a server for n_dfas loaded DFAs (all on the current device; the array is copied, the
 * DFAs stay owned by the caller and must outlive the server).  Allocates the arenas, streams
 * and threads.  Errors: INVALID_ARG, OOM, CUDA. */
int parem_server_create(parem_dfa* const* dfas, uint32_t n_dfas, const parem_server_opts* opts,
                        parem_server** out);

/* Queue n requests (host array, copied).  Errors: INVALID_ARG (a bad DFA index or null text;
 * nothing is queued). */
int parem_server_submit(parem_server* srv, const parem_request* reqs, uint32_t n);

/* Move up to max finished responses into out (in completion order); *n_out is their number.
 * Waits up to wait_ns for the first one (0 = do not wait).  Errors: INVALID_ARG. */
int parem_server_poll(parem_server* srv, parem_response* out, uint32_t max, uint32_t* n_out, int64_t wait_ns);

/* Wait until every submitted request has a response waiting to be polled. */
int parem_server_drain(parem_server* srv);

/* Open-loop trace replay: submit reqs[i] at (start + reqs[i].arrival_ns) from a library thread,
 * where start is the time of the call, and wait for all of them; out[i] is reqs[i]'s response
 * (the tags are replaced by i).  Responses queued before the call are kept for
 * parem_server_poll.  Errors: INVALID_ARG, and the first failing request's status is not an
 * error of the call (read out[i].status). */
int parem_server_replay(parem_server* srv, const parem_request* reqs, uint32_t n, parem_response* out);

int parem_server_get_stats(const parem_server* srv, parem_server_stats* out);

/* Stop the threads after the submitted requests have been served, and free the server. */
void parem_server_free(parem_server* srv);

/* The steady clock the server stamps responses with (nanoseconds). */
int64_t parem_clock_ns(void);

/* Plan and kernel times of the last scan issued on (current device, stream); waits for the
 * recorded events.  Errors: INVALID_ARG (no scan yet), CUDA. */
int parem_last_stats(void* stream, parem_stats* out);

/* Release the scratch memory cached for (current device, stream).  Errors: CUDA. */
int parem_release_scratch(void* stream);

/* Message for a status code. */
const char* parem_strerror(int status);

/* Library version "major.minor.patch". */
const char* parem_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PAREM_H */
