/*
 * propagate.h — C ABI of the GB300 (sm_103a) implementation of PROPAGATE
 * (Amati, Cruciani, Pasquini, Vocca, Angelini: "PROPAGATE: a seed propagation
 * framework to compute Distance-based metrics on Very Large Graphs").
 *
 * The method (Sec. 4): every node u carries a Boolean signature Sig(u) of s
 * bits, bit i set iff seed x_i has reached u. One synchronous round computes
 *     Sig'(v) = Sig(v) OR ( OR over in-neighbours u of v of Sig(u) )
 * and the popcount of Sig'(v) XOR Sig(v) per seed gives the nodes at distance
 * exactly t from each seed (the "collisions" of Sec. 4). PROPAGATE-P
 * (Algorithm 1, Sec. 4.1) moves all s bits per round; PROPAGATE-S
 * (Algorithm 2, Sec. 4.2) handles one seed per 1-bit plane, pulling only into
 * unset nodes and stopping a node's scan at the first set in-neighbour. From
 * the per-round counts follow the neighbourhood function, diameter,
 * effective diameter, average distance, reachable pairs and connectivity
 * rate (Sec. 3).
 *
 * Conventions shared by every entry point:
 *  - A graph is a CSR over IN-edges: row v lists every u with an arc u -> v
 *    (the arcs a pull reads). Counts are balls grown forward from each seed
 *    along arcs. An undirected graph is passed symmetrised.
 *  - Seed i owns bit (i mod 64) of signature word floor(i / 64).
 *  - Every call is ordered on the CUDA stream it is given (NULL = the legacy
 *    default stream) and returns once its host outputs are written.
 *  - Calls on one pg_graph are serialised by the library; different graphs
 *    may be used from different host threads concurrently.
 *  - No entry point aborts the process. Errors are returned as pg_status and
 *    leave the graph usable; pg_strerror names them.
 */
#ifndef PROPAGATE_H
#define PROPAGATE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PG_OK = 0,
  PG_EINVAL = -1,      /* bad argument: CSR, seeds, sizes, options */
  PG_ENOMEM = -2,      /* device or pinned host memory could not be had */
  PG_ECUDA = -3,       /* a CUDA runtime call failed */
  PG_ETIMEOUT = -4,    /* a bounded device-side wait expired */
  PG_EDEVICE = -5,     /* the device reported an inconsistent state */
  PG_ECANCELLED = -6,  /* the request was cancelled */
  PG_ERANGE = -7,      /* more rounds than the caller's max_rounds */
  PG_ETOOBIG = -8      /* problem larger than the fixed scratch of
                          pg_propagate_p_noalloc */
} pg_status;

/* Opaque graph handle: device-resident CSR (in-edges and, for directed
 * graphs, out-edges), cached per-call workspace. Library-owned. */
typedef struct pg_graph pg_graph;

/* pg_graph_from_csr flags */
#define PG_DEVICE_PTRS 1u /* row_ptr and col are device pointers */
#define PG_BORROW 2u      /* with PG_DEVICE_PTRS: use the caller's arrays in
                             place; they must outlive the graph */
#define PG_REVERSE 4u     /* pull along the other direction: the counts are
                             then balls grown backward, the nodes that reach
                             each seed (the direction Algorithm 1 literally
                             iterates, Sig(u) |= Sig(v) for u -> v); the
                             library pulls over the out-edge transpose it
                             builds. Directed graphs only (undirected graphs
                             are their own transpose). */
#define PG_RELABEL 8u     /* renumber the nodes internally, high in-degree
                             first (buckets of 16 per octave of degree, each
                             in the original order): the most gathered rows
                             then share cache lines and stay in L2. Seeds are
                             still given, and counts returned, in the
                             caller's ids and order; every output is
                             unchanged. Without PG_RELABEL or PG_KEEP_ORDER
                             the library relabels graphs of at least 2^16
                             nodes whose largest in-degree is at least 16
                             times the mean (skewed, power-law degrees) */
#define PG_KEEP_ORDER 16u /* never relabel */
#define PG_HOST_CSR 32u   /* keep the arc arrays (column indices, the out-edge
                             transpose's, and the dense rounds' sliced-ELL
                             copy) in pinned host memory, read by the kernels
                             over the CPU-GPU link, so that a graph whose
                             arcs exceed device memory can still run: only
                             row pointers, signatures, bitmaps and lists
                             stay on the device. Not with PG_BORROW */

/*
 * Per-round, per-seed counts. Caller-owned host buffers.
 *  counts   [ (max_rounds+1) * s ]: counts[t*s + i] = number of nodes at
 *           distance exactly t from seed i (row 0 is all ones). Rows
 *           0..rounds are written.
 *  m_active [ max_rounds + 2 ] (may be NULL): m_active[t] = sum of the
 *           in-degrees of the nodes that round t had to revisit: nodes with
 *           a zero bit (skip rule in the proof of Thm. 1) and an in-neighbour
 *           that changed in round t-1. Entry 0 is 0; entry rounds+1 is the
 *           final sweep that found no change. For PROPAGATE-S the entry is
 *           summed over the seed passes.
 *  rounds   out: T = the last round with a new (seed, node) pair, i.e. the
 *           diameter lower bound Delta_LB of Algorithm 1.
 */
typedef struct {
  int32_t s;          /* in: number of seeds (columns of counts) */
  int32_t max_rounds; /* in: capacity, see above; pg_query_rounds_bound */
  int32_t rounds;     /* out */
  int32_t reserved;
  uint32_t *counts;   /* out, host */
  uint64_t *m_active; /* out, host, optional */
} pg_counts;

/* Schedule options. Every choice gives bit-identical counts; they change
 * only how the rounds are executed. Zero-initialise and call
 * pg_default_options, or pass NULL for defaults. */
typedef struct {
  int32_t direction;        /* PG_DIR_AUTO: per round, a frontier-driven
                               (sparse) sweep when the frontier's out-arcs are
                               few, a full (dense) sweep otherwise */
  float dense_threshold;    /* AUTO: dense when frontier out-arcs > this * m
                               (0 = library default) */
  int32_t group_lanes;      /* lanes sharing one work piece (1..32, power of
                               two); a piece is group_lanes x 8 in-arcs for
                               s <= 128, x 4 for s <= 256, x 2 above, and
                               longer rows are split into
                               pieces combined with atomic OR; 0 = the
                               smallest group whose piece covers the mean
                               in-degree */
  int32_t test_changed;     /* an in-neighbour u adds to v only the bits u
                               gained in the previous round (its delta, zero
                               if u did not change). 1: test u's changed bit
                               before reading its delta; 2: always read the
                               delta; 3: decide per round, testing while the
                               previous round's frontier out-arcs are below
                               half of all arcs; 0 (auto): 3 when the deltas
                               exceed 64 MiB (n x words per row x 8 bytes),
                               else 2 (a packed batch: 1 instead of 3) */
  int32_t planes_per_pass;  /* PROPAGATE-S: seeds per pass, 1..64; 0 = 64 */
  int32_t use_graphs;       /* 1: the round loop is one CUDA graph with a
                               device-driven while node (no host round trip
                               per round); 0: plain launches in batches */
  int32_t timing;           /* 1: record CUDA events around every kernel
                               launch (plain launches) for pg_last_stats */
  int32_t window_rows;      /* rows of per-round counters kept on the device
                               before they are copied out; 0 = auto */
  int32_t words_per_thread; /* signature words one lane gathers per in-arc
                               (1, 2, 4 or 8; a row of more words is swept in
                               chunks of this many); 0 = the row's words
                               rounded up to 1, 2, 4 or 8 */
  int32_t wide_rows;        /* rows of more than 8 words (s > 512): 0 or 1 =
                               a warp per row piece, its lanes spread over
                               the words (one contiguous read per gathered
                               neighbour); 2 = lanes over 8-word chunks as
                               for narrower rows (words_per_thread applies) */
  int32_t passes_together;  /* PROPAGATE-S: passes run as one propagation over
                               that many copies of the graph side by side
                               (passes never exchange bits), as far as a
                               quarter of the free device memory holds the
                               copies; 1 = one pass at a time; 0 = automatic:
                               when passes do not run as words (pass_words),
                               as many as keep the copies under 2^24 arcs
                               (small graphs, where one pass cannot fill the
                               GPU) */
  int32_t pass_words;       /* PROPAGATE-S with 64 planes per pass: passes
                               run side by side as the words of one
                               signature over the same graph (word k = pass
                               k's 64 one-bit planes; passes never exchange
                               bits, and counts, rounds and m_active are each
                               pass's own). 1 = one word per node; K >= 2 =
                               up to K passes per propagation; 0 = all of
                               them. Either as far as a quarter of the free
                               device memory holds four buffers of n x 8K
                               bytes; copies of the graph (passes_together)
                               then serve only passes of fewer planes or an
                               explicit passes_together > 1 */
  int32_t tma_gather;       /* dense rounds of rows of 4 or 8 words (s of 129
                               to 512, or PROPAGATE-S passes as 4 or 8
                               words): 2 = the neighbours' delta rows are
                               copied into shared memory by the tensor memory
                               accelerator (four rows per tile::gather4 copy,
                               several steps in flight per warp) instead of
                               loaded by each lane; 0 or 1 = per-lane loads
                               (the default: they measured faster on a 2^26-
                               node graph with 8-word rows) */
  int32_t sparse_push;      /* sparse rounds: 0 (default) or 2 = push, each
                               row that changed in the previous round ORs
                               its delta into its out-neighbours with
                               atomics (their claims for m_active made on
                               the way, per pass for PROPAGATE-S passes run
                               as words), where it applies: rows of up to 8
                               words (s <= 512, or up to 8 passes as words)
                               gathered whole, one graph or a packed batch
                               (pg_batch_run: its graphs below their dense
                               threshold push while the others are swept
                               whole); 1 = pull, the post kernel claims the
                               frontier's out-neighbours and the pull
                               gathers their in-arcs (always for rows above
                               8 words) */
} pg_options;

#define PG_DIR_AUTO 0
#define PG_DIR_DENSE 1  /* every round a full sweep over unsaturated nodes */
#define PG_DIR_SPARSE 2 /* every round only the nodes reached by the frontier */

typedef struct {
  int32_t diameter;              /* Delta_LB = T (Alg. 1) */
  int32_t eff_diameter;          /* min k: R[k] >= tau R[T] (Sec. 3, Alg. 1) */
  double eff_diameter_interp;    /* (k-1) + (tau R[T]-R[k-1])/(R[k]-R[k-1]); 0 if k = 0 */
  double avg_distance;           /* sum_r r (R[r]-R[r-1]) / (R[T] - s): pairs u != v */
  double avg_distance_incl_self; /* same numerator / R[T] (Alg. 1's division) */
  double connectivity_rate;      /* (R[T] - s) / (s (n-1)) (Sec. 3 alpha) */
  double reachable_pairs;        /* (n/s) R[T] (Alg. 1), self-pairs included */
  uint64_t R_last;               /* R[T] over the s seeds */
  uint64_t dist_sum;             /* sum_r r (R[r]-R[r-1]) */
} pg_metrics_out;

/*
 * Progressive sampling. Sec. 4.2 notes that the seed-by-seed variant can keep
 * adding seeds until the estimates settle, and Sec. 6 lists this progressive
 * sampling as one of its uses; the paper gives no stopping rule. Thm. 3 puts
 * the sample a fixed accuracy needs at the order ln n / eps^2. This call
 * draws seeds uniformly without replacement from a seeded SplitMix64 stream
 * (its first distinct values, so a smaller sample is a prefix of a larger
 * one), runs PROPAGATE-P on blocks of `block` seeds, appends each block's
 * per-seed count columns (seeds never interact, so they equal one call over
 * all drawn seeds), and stops at ceil(ln n / eps^2) seeds (capped at n; the
 * constant 1 is this library's reading) or, with stable_tol > 0, as soon as
 * the average distance and the interpolated effective diameter (tau = 9/10)
 * both moved by less than stable_tol (relative) over two consecutive blocks.
 *  seeds    host int32[out->s] out: the drawn seeds in draw order
 *  s_drawn  out: seeds drawn (columns of counts written)
 *  out      out->s (in) = the caller's column capacity, at least
 *           min(n, ceil(ln n / eps^2)); counts[t * out->s + i] for i <
 *           *s_drawn as pg_counts (zero elsewhere); m_active (optional) sums
 *           each block's own m_active; out->rounds = the largest T
 *  history  pg_metrics_out[max_history] (may be NULL if max_history = 0):
 *           the metrics over all seeds drawn after each block
 *  blocks   out (may be NULL): blocks run
 * Errors: PG_EINVAL (arguments, eps <= 0, too few columns), PG_ERANGE (a
 * block needed more than out->max_rounds rounds), else as pg_propagate_p.
 */
pg_status pg_progressive(pg_graph *g, double eps, int32_t block, double stable_tol,
                         uint64_t rng_seed, int32_t *seeds, int32_t *s_drawn, pg_counts *out,
                         pg_metrics_out *history, int32_t max_history, int32_t *blocks,
                         const pg_options *opt, void *stream);

/* Work and timing of the last propagate call on a graph (for benchmarks). */
typedef struct {
  int32_t sweeps;            /* rounds executed, the final empty one included */
  int32_t passes;            /* seed passes (1 for PROPAGATE-P) */
  int32_t dense_rounds;      /* rounds run as full sweeps */
  int32_t launches;          /* kernels launched by the call */
  uint64_t m_active_total;   /* sum over rounds (and passes) of m_active */
  uint64_t arcs_scanned;     /* column indices read by the pull kernel */
  uint64_t rows_gathered;    /* neighbour signatures ORed by the pull kernel */
  uint64_t items;            /* row pieces visited by the pull kernel */
  uint64_t changed_rows;     /* sum over rounds of rows that changed */
  uint64_t frontier_arcs;    /* sum over sparse rounds of the frontier's out-arcs */
  int32_t words_per_row;     /* 64-bit signature words per node (padded) */
  int32_t group_lanes;       /* lanes per work piece used */
  double ms_pull;            /* with timing=1: summed event time per kernel */
  double ms_post;
  double ms_init;
  int32_t pull_launches;
  int32_t post_launches;
  int32_t test_changed;      /* 1 if changed bits were tested before gathers */
  int32_t words_per_gather;  /* signature words one lane gathers per arc (the
                                pull instantiation k_pull<words, lanes>); 0 =
                                the wide-row kernel (a warp per piece) */
  uint64_t seed_edge_traversals; /* sum over rounds and active rows of
                               s x in-degree (the benchmark's work measure;
                               s of the row's own graph in a batch) */
  int32_t pass_words;        /* PROPAGATE-S: passes run side by side as the
                                words of one signature (the pull instantiation
                                k_pull<words, lanes, 1>); 1 otherwise */
  int32_t dense_tma;         /* 1 if dense rounds gathered deltas by TMA
                                (k_pull_tma<words, pass_words>) */
  uint64_t active_rows;      /* sum over rounds of |A_t|, the rows a round had
                                to revisit (those m_active sums the in-degrees
                                of); PROPAGATE-S: summed over passes */
} pg_stats;

/* Message for a status code (static storage). */
const char *pg_strerror(pg_status st);

/* Library version string. */
const char *pg_version(void);

/* Fills *opt with the defaults. */
void pg_default_options(pg_options *opt);

/*
 * Builds a graph from a CSR over in-edges (Sec. 4 recurrence: row v is the
 * set of nodes whose ball is unioned into v's).
 *  row_ptr  int64[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = m
 *  col      int32[m], each in [0, n), strictly increasing within a row
 *  directed 1: general digraph (the library builds the out-edge transpose);
 *           0: the caller asserts the CSR is symmetric (in = out)
 *  flags    PG_DEVICE_PTRS / PG_BORROW / PG_REVERSE; host arrays are copied
 *  stream   cudaStream_t for the copies and validation kernels
 * Errors: PG_EINVAL for n < 1, n >= 2^27 or m >= 2^37 (the largest graph
 * whose rounds the kernels can count: one 64-bit counter holds a round's
 * changed rows in 27 bits and their out-arcs in 37), m < 0, or a malformed
 * CSR (checked on the device); PG_ENOMEM; PG_ECUDA.
 */
pg_status pg_graph_from_csr(const int64_t *row_ptr, const int32_t *col, int64_t n, int64_t m,
                            int directed, unsigned flags, void *stream, pg_graph **out);

/* Frees the graph and its cached workspace. NULL is allowed. */
void pg_graph_free(pg_graph *g);

/* *relabelled = 1 if the library renumbered g's nodes internally
 * (PG_RELABEL, or by default on a skewed graph), else 0. */
pg_status pg_graph_is_relabelled(const pg_graph *g, int32_t *relabelled);

/*
 * Graph generators on the device. The paper measures on real graphs
 * (Table 1); these are the seeded synthetic stand-ins of the same classes,
 * drawn on the GPU from one counter-based SplitMix64 stream (draw i of stream
 * k under a seed), so that they equal, arc for arc, what any implementation
 * of the same definitions produces (the tests compare with the host
 * generators):
 *  PG_GEN_ER    undirected G(n, M), M = round(n avg_degree / 2) uniform
 *               pairs with replacement (draws 2i, 2i+1 of stream 0)
 *  PG_GEN_RMAT  2^scale nodes, round(edge_factor 2^scale) edges, each by
 *               `scale` quadrant choices with probabilities (a, b, c, 1-a-b-c)
 *               quantised to 16 bits, four levels per draw of stream 1; no
 *               noise, no permutation; directed keeps src -> dst, else
 *               symmetrised
 *  PG_GEN_GRID  rows x cols 4-neighbour lattice, node (r, c) = r cols + c,
 *               edge i deleted when draw i of stream 2 < p_delete 2^64
 * Self-loops are dropped and duplicates removed. The CSR over in-edges is
 * built on the device (a radix sort of the arc keys, a scan for the unique
 * ones) and becomes the graph as pg_graph_from_csr would make it (flags as
 * there, except PG_DEVICE_PTRS, PG_BORROW and PG_HOST_CSR). Errors: PG_EINVAL
 * (sizes, probabilities; n >= 2^27 as for pg_graph_from_csr), PG_ENOMEM,
 * PG_ECUDA.
 */
#define PG_GEN_ER 0
#define PG_GEN_RMAT 1
#define PG_GEN_GRID 2
typedef struct {
  int32_t kind;        /* PG_GEN_ER, PG_GEN_RMAT or PG_GEN_GRID */
  int32_t directed;    /* PG_GEN_RMAT only: 1 = arcs src -> dst, 0 = symmetrised */
  uint64_t seed;
  int64_t n;           /* PG_GEN_ER: nodes */
  double avg_degree;   /* PG_GEN_ER */
  int32_t scale;       /* PG_GEN_RMAT: 2^scale nodes (1..26) */
  int32_t reserved;
  double edge_factor;  /* PG_GEN_RMAT */
  double a, b, c;      /* PG_GEN_RMAT quadrant probabilities */
  int64_t rows, cols;  /* PG_GEN_GRID */
  double p_delete;     /* PG_GEN_GRID */
} pg_generator;
pg_status pg_graph_generate(const pg_generator *gen, unsigned flags, void *stream,
                            pg_graph **out);

/* Copies g's CSR over in-edges, as the kernels read it (the library's
 * internal node ids: the caller's unless the graph was relabelled), into
 * row_ptr[n+1] and col[m] (host or device; the call returns when they are
 * written). Errors: PG_EINVAL, PG_ECUDA. */
pg_status pg_graph_copy_csr(const pg_graph *g, int64_t *row_ptr, int32_t *col, void *stream);

/* n and m of a graph. */
pg_status pg_graph_info(const pg_graph *g, int64_t *n, int64_t *m);

/* A safe max_rounds: every eccentricity is at most n - 1. */
pg_status pg_query_rounds_bound(const pg_graph *g, int32_t *max_rounds);

/*
 * PROPAGATE-P (Algorithm 1, Sec. 4.1): all s seeds diffuse synchronously, s
 * bits per node; stops at the first round with no new bit (do ... while
 * Count > 0). seeds: host int32[s], distinct, in [0, n). out->s must equal s;
 * out->counts and out->m_active sized by out->max_rounds as documented.
 * Errors: PG_EINVAL (s < 1, duplicate or out-of-range seeds, bad sizes),
 * PG_ERANGE (more than max_rounds productive rounds; rows 0..max_rounds are
 * written and out->rounds = max_rounds + 1), PG_ENOMEM, PG_ECUDA.
 */
pg_status pg_propagate_p(pg_graph *g, const int32_t *seeds, int32_t s, pg_counts *out,
                         const pg_options *opt, void *stream);

/*
 * PROPAGATE-S (Algorithm 2, Sec. 4.2): seeds are processed in passes of
 * planes_per_pass independent 1-bit planes (plane k of a node is bit k of its
 * word); in each round only nodes with an unset plane pull, and a node whose
 * planes are all set is not scanned again (Algorithm 2's break at the first
 * set in-neighbour, with one plane per pass, becomes this skip when a node's
 * in-neighbours are read in parallel pieces). Passes are independent: by
 * default they run side by side, as the words of one signature over the
 * graph (pg_options.pass_words) or on copies of it (passes_together), each
 * pass keeping its own counts, rounds and m_active; pass_words = 1 with
 * passes_together = 1 runs them one after another, Algorithm 2's schedule
 * and memory footprint. The counts are per seed and identical to
 * PROPAGATE-P's (Sec. 5, both algorithms give the same results). Arguments
 * and errors as pg_propagate_p; m_active is each pass's own, summed over
 * the passes.
 */
pg_status pg_propagate_s(pg_graph *g, const int32_t *seeds, int32_t s, pg_counts *out,
                         const pg_options *opt, void *stream);

/*
 * Metrics of Sec. 3 and of the last steps of Algorithm 1 from counts
 * (rows 0..c->rounds), for an n-node graph and threshold tau = tau_num /
 * tau_den in (0, 1] (the paper uses 9/10). Host-only, FP64 divisions of exact
 * 64-bit integer sums; tau is applied by integer cross-multiplication.
 * Errors: PG_EINVAL.
 */
pg_status pg_metrics(const pg_counts *c, int64_t n, int32_t tau_num, int32_t tau_den,
                     pg_metrics_out *out);

/* Work counters and (with timing=1) kernel times of the last propagate call
 * on g. */
pg_status pg_last_stats(const pg_graph *g, pg_stats *out);

/*
 * Autotuner. The paper fixes no schedule (its loops are sequential Java);
 * the GPU's free parameters are the lanes per work piece (group_lanes), the
 * signature words a lane gathers per arc (words_per_thread) and the
 * frontier density at which a round becomes a full sweep (dense_threshold),
 * whether changed bits are tested before delta gathers (test_changed) and
 * whether sparse rounds push or pull (sparse_push). pg_autotune
 * times PROPAGATE-P (algorithm PG_ALG_P) or PROPAGATE-S (PG_ALG_S) on g
 * with these seeds under candidate values, one
 * parameter at a time starting from *inout (coordinate descent; a candidate
 * replaces the current value when it is at least 2% faster), and writes the
 * fastest options back to *inout. Every candidate's counts are compared
 * with the first run's; a difference returns PG_EDEVICE. max_trials bounds
 * the timed propagations (each candidate is run three times, the fastest
 * kept).
 * Errors: as pg_propagate_p.
 */
typedef struct {
  int32_t trials;       /* propagations run */
  int32_t improved;     /* accepted changes */
  double default_ms;    /* best time of the starting options */
  double best_ms;       /* best time of the returned options */
} pg_tune_report;

#define PG_ALG_P 0 /* PROPAGATE-P (Algorithm 1) */
#define PG_ALG_S 1 /* PROPAGATE-S (Algorithm 2): also tunes passes_together */
pg_status pg_autotune(pg_graph *g, const int32_t *seeds, int32_t s, int32_t algorithm,
                      int32_t max_trials, pg_options *inout, pg_tune_report *report,
                      void *stream);

/*
 * Allocation-free PROPAGATE-P. The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory while they
 * run (for example a serving process that reserves all of its device memory
 * at start-up, or a latency-critical loop that cannot take the device-wide
 * synchronisation an allocation may cause). It computes the same counts as
 * pg_propagate_p, with every dense-round intermediate held in one fixed
 * file-scope device array of PG_NOALLOC_SCRATCH_BYTES that each GPU loading
 * the library keeps until the process exits; it calls no cudaMalloc or
 * cudaFree.
 *  row_ptr, col  device pointers, CSR over in-edges as for pg_graph_from_csr
 *                (checked on the device; sortedness is not required)
 *  seeds         host int32[s], distinct, in [0, n); s <= PG_NOALLOC_MAX_SEEDS
 *  counts        device uint32[(max_rounds+1) * s], caller-allocated; zeroed
 *                and filled like pg_counts.counts
 *  rounds        host out: T as in pg_counts.rounds
 *  stream        cudaStream_t; the call returns when the counts are written
 * Limits: 4 * n * ceil(s/64) 64-bit words plus a small header must fit the
 * scratch (with s <= 64, n up to about one million); larger problems return
 * PG_ETOOBIG. Errors: PG_EINVAL (arguments, seeds, CSR), PG_ERANGE (rows
 * 0..max_rounds written, *rounds = max_rounds + 1), PG_ECUDA (a launch or
 * copy failed). The call waits on the stream after validation and after every
 * round (it reads the round's changed flag back to the host).
 * Because it waits on the stream every round, the call cannot be captured
 * into a CUDA graph: do not make it while its stream (or, for the legacy
 * stream, any stream) is capturing. The first call on a device also looks
 * up the array's device address (once per device). All calls share
 * the array and each clears what it uses; calls whose GPU work overlaps (on
 * different streams) race on it, so order them on one stream.
 */
#define PG_NOALLOC_SCRATCH_BYTES (32u << 20)
#define PG_NOALLOC_MAX_SEEDS 1024
pg_status pg_propagate_p_noalloc(const int64_t *row_ptr, const int32_t *col, int64_t n,
                                 int64_t m, const int32_t *seeds, int32_t s, uint32_t *counts,
                                 int32_t max_rounds, int32_t *rounds, void *stream);

/*
 * Batched PROPAGATE-P over many independent graphs. Sec. 4 notes that the
 * work of a round splits over nodes without interaction; graphs that share
 * nothing split the same way, so a batch packs the graphs of one signature
 * width class (ceil(s/64) words rounded to 1, 2, 4 or a multiple of 8) into
 * one disjoint union and runs each class as a single PROPAGATE-P: one pull
 * and one post launch per round for all of its graphs. Each graph's counts
 * equal what pg_propagate_p gives for it alone (its bits never leave its own
 * nodes), and so does its m_active (the kernels add each active row's
 * in-degree to its own graph's slot of the round as well). A graph of at
 * least 2^16 nodes whose four signature arrays (n x
 * words x 8 bytes each) fill half of L2 or more runs alone instead, as
 * pg_propagate_p would run it: it fills the GPU by itself, and alone it
 * keeps part of its arrays in L2 from round to round. The paper runs one
 * graph per call; batching is this library's addition for workloads of
 * many small graphs.
 */
typedef struct pg_batch pg_batch;

typedef struct {
  int32_t graphs;                /* graphs in the batch */
  int32_t groups;                /* propagations: one per width class of
                                    packed graphs, one per graph run alone */
  int32_t sweeps;                /* rounds of the longest class */
  int32_t launches;              /* kernels launched over all classes */
  uint64_t seed_edge_traversals; /* sum over graphs of their own
                                    pg_stats.seed_edge_traversals */
} pg_batch_stats;

/* New empty batch. Errors: PG_EINVAL (out NULL). */
pg_status pg_batch_create(pg_batch **out);

/* Frees the batch, its packed device graphs and stored results. NULL is
 * allowed. */
void pg_batch_free(pg_batch *b);

/*
 * Adds a graph (host CSR over in-edges as for pg_graph_from_csr, copied) and
 * its seeds (host int32[s], distinct, in [0, n)). *index (may be NULL)
 * receives the graph's position, used by pg_batch_result. Adding after a run
 * repacks the batch on the next run. Errors: PG_EINVAL (arguments, seeds,
 * row_ptr ends, n >= 2^27 or m >= 2^37 as for pg_graph_from_csr); the CSR's
 * columns are checked on the device at the run. A width class whose graphs
 * together pass those sizes is packed into several unions.
 */
pg_status pg_batch_add(pg_batch *b, const int64_t *row_ptr, const int32_t *col, int64_t n,
                       int64_t m, int directed, const int32_t *seeds, int32_t s,
                       int32_t *index);

/*
 * Runs every graph of the batch to its last productive round and keeps each
 * graph's counts on the host. The groups (packed width classes and graphs
 * run alone) run up to four at a time (pg_batch_set_streams), each on a
 * stream the batch owns,
 * driven by a host thread of its own; they start after the work already
 * queued on `stream`, and the call returns when all of them are done. opt
 * as for pg_propagate_p (planes_per_pass is ignored); NULL = the options
 * pg_batch_tune chose, else the defaults. Errors: PG_EINVAL (empty batch,
 * malformed CSR), PG_ENOMEM, PG_ECUDA; on error no result of this run is
 * kept.
 */
pg_status pg_batch_run(pg_batch *b, const pg_options *opt, void *stream);

/*
 * Copies graph index's counts of the last run into out (out->s must equal
 * the graph's s; rows 0..min(T, out->max_rounds)) and, when out->m_active is
 * set, its own m_active as pg_propagate_p writes it (entries
 * 0..min(T + 1, out->max_rounds + 1), zero beyond). Errors: PG_EINVAL (no run,
 * bad index or s), PG_ERANGE (T > out->max_rounds; out->rounds = T).
 */
pg_status pg_batch_result(pg_batch *b, int32_t index, pg_counts *out);

/* Work counters of the last pg_batch_run. */
pg_status pg_batch_get_stats(pg_batch *b, pg_batch_stats *out);

/*
 * Tunes each group of the batch as pg_autotune does (each timed run is a
 * full run of that group; counts compared across candidates) and keeps the
 * chosen options per group; pg_batch_run with opt == NULL then uses them.
 * report (may be NULL) receives the sums over groups.
 */
pg_status pg_batch_tune(pg_batch *b, int32_t max_trials, pg_tune_report *report, void *stream);

/* Groups pg_batch_run runs at once (1..16, default 4), each on its own
 * stream; 1 runs them one after another (kernel times of a group then
 * measure that group alone). Errors: PG_EINVAL (b NULL, streams out of
 * range). */
pg_status pg_batch_set_streams(pg_batch *b, int32_t streams);

/* pg_stats of group `group` in the last pg_batch_run (kernel times with
 * opt->timing = 1). Groups are numbered by increasing width; within a width
 * class the packed graphs come first, then the graphs run alone. Errors:
 * PG_EINVAL (no such group or no run). */
pg_status pg_batch_group_stats(pg_batch *b, int32_t group, pg_stats *out);

/* Options a group of the batch runs with (tuned, else the defaults); groups
 * are numbered as for pg_batch_group_stats after the first run or tune;
 * *graphs (may be NULL) receives the group's graph count. Errors: PG_EINVAL
 * (no such group). */
pg_status pg_batch_get_options(pg_batch *b, int32_t group, pg_options *out, int32_t *graphs);

/*
 * Serving loop. The paper runs one query per call; this is the library's
 * request loop for many metric queries on resident graphs (the Sec. 4
 * remark that seeds are independent is what lets queries share a run).
 *
 * The server keeps registered graphs on the device. A request names a graph
 * and a seed set and is answered with the counts pg_propagate_p would give
 * for it alone (m_active is not kept per request). `slots` worker threads,
 * each with its own CUDA stream and workspace, take queued requests as soon
 * as a slot and device memory are free (continuous batching): a free slot
 * takes the oldest request that fits the memory budget and merges into the
 * same propagation the other queued requests on that graph (up to merge_max
 * requests and merge_max_seeds seeds; seeds of different requests are
 * independent bit columns and may coincide) and, with cross_graph, queued
 * requests on other graphs of the same signature width: those graphs run
 * as one disjoint union, as a batch does (pg_batch_*), built on the device
 * from the resident copies for that propagation. Propagations on different
 * slots run concurrently on the device.
 *
 * Memory admission: resident graphs (CSR, out-CSR, sliced-ELL copy) plus
 * every slot's workspace and cached piece lists stay within hbm_budget.
 * A request is charged its workspace, about 32 bytes per node per 64 seeds
 * (four signature buffers) plus the frontier lists and its counts window. A
 * request that cannot fit an idle server is refused at submission
 * (PG_ENOMEM); others wait until memory frees up, idle slots first dropping
 * their caches.
 *
 * All calls are thread-safe. Requests run on the device current when the
 * server was created; the server's calls must be made with that device
 * current.
 */
typedef struct pg_server pg_server;

typedef struct {
  int32_t slots;            /* concurrent propagations (1..64; default 4) */
  int32_t merge_max;        /* most requests merged into one propagation (16) */
  int32_t merge_max_seeds;  /* most seeds of a merged propagation (8192) */
  int32_t cross_graph;      /* 1 (default): a propagation may also merge
                               queued requests on other graphs of the same
                               signature width (1, 2, 4 or a multiple of 8
                               words), run as one packed union of those
                               graphs (up to 2^22 nodes, each graph its own
                               kind of round); 0: requests on one graph only */
  int64_t hbm_budget;       /* device bytes for graphs + workspaces; 0 = 90% of
                               the memory free at creation */
  pg_options opt;           /* options of every propagation (timing ignored;
                               window_rows 0 = 256) */
} pg_server_config;

typedef enum {
  PG_REQ_QUEUED = 0,
  PG_REQ_RUNNING = 1,
  PG_REQ_DONE = 2,
  PG_REQ_FAILED = 3,
  PG_REQ_CANCELLED = 4
} pg_request_state;

typedef struct {
  int32_t state;      /* pg_request_state */
  int32_t status;     /* PG_OK, or the error of a failed / cancelled request */
  int32_t rounds;     /* T once done */
  int32_t s;          /* seeds of the request */
  int32_t graph;      /* graph id */
  int32_t merged;     /* requests in the propagation that served it */
  int64_t footprint;  /* device bytes its slot was charged */
  int64_t submit_ns;  /* steady-clock times of submission, start, end */
  int64_t start_ns;
  int64_t done_ns;
} pg_request_info;

typedef struct {
  int64_t submitted, completed, failed, cancelled;
  int64_t propagations;           /* runs on the device (merged requests share one) */
  int64_t resident_bytes;         /* registered graphs */
  int64_t inflight_bytes;         /* slots' workspaces and caches now */
  int64_t peak_bytes;             /* most resident + slot bytes charged at once */
  int64_t budget_bytes;           /* the admission budget */
  int32_t graphs, queued, running, reserved;
  uint64_t seed_edge_traversals;  /* summed over propagations */
  int64_t gpu_launches;           /* kernels the propagations launched */
} pg_server_stats;

/* Fills *cfg with the defaults. */
void pg_server_default_config(pg_server_config *cfg);

/* Starts a server on the current device (cfg NULL = defaults). Errors:
 * PG_EINVAL (config), PG_ECUDA. */
pg_status pg_server_create(const pg_server_config *cfg, pg_server **out);

/* Cancels queued requests, lets running ones finish, frees everything.
 * NULL is allowed. */
void pg_server_destroy(pg_server *srv);

/*
 * Registers a graph (host CSR over in-edges, as for pg_graph_from_csr; copied
 * to the device). *graph_id receives its id. Errors: PG_EINVAL (CSR),
 * PG_ENOMEM (budget or device memory), PG_ECUDA.
 */
pg_status pg_server_add_graph(pg_server *srv, const int64_t *row_ptr, const int32_t *col,
                              int64_t n, int64_t m, int directed, int32_t *graph_id);

/* Unregisters a graph with no queued or running request (else PG_EINVAL). */
pg_status pg_server_remove_graph(pg_server *srv, int32_t graph_id);

/*
 * Queues a request: seeds host int32[s], distinct, in [0, n) of the graph;
 * copied. Returns at once with *request_id. Errors: PG_EINVAL (graph, seeds),
 * PG_ENOMEM (cannot fit the budget even alone).
 */
pg_status pg_server_submit(pg_server *srv, int32_t graph_id, const int32_t *seeds, int32_t s,
                           int64_t *request_id);

/* State and times of a request (info required). */
pg_status pg_server_poll(pg_server *srv, int64_t request_id, pg_request_info *info);

/* Blocks until the request is done, failed or cancelled, or timeout_ms
 * passes (< 0: no limit; PG_ETIMEOUT then). info may be NULL. */
pg_status pg_server_wait(pg_server *srv, int64_t request_id, int32_t timeout_ms,
                         pg_request_info *info);

/*
 * Copies a finished request's counts into out (out->s must equal its s; rows
 * 0..min(T, out->max_rounds); m_active zero-filled) and releases the request.
 * A failed or cancelled request returns its status and is released. Errors:
 * PG_EINVAL (unknown or unfinished request, bad out), PG_ERANGE (T >
 * out->max_rounds; the request is kept so that a larger buffer can be
 * offered).
 */
pg_status pg_server_result(pg_server *srv, int64_t request_id, pg_counts *out,
                           pg_request_info *info);

/* Cancels a queued request; a running one completes on the device and its
 * result is dropped (state PG_REQ_CANCELLED). */
pg_status pg_server_cancel(pg_server *srv, int64_t request_id);

/* Counters of the server. */
pg_status pg_server_get_stats(pg_server *srv, pg_server_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* PROPAGATE_H */
