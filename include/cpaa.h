/*
 * cpaa.h -- C ABI of the GB300 (sm_103a) CPAA PageRank library.
 *
 * CPAA (Zhang, Tang, Yao, Zhang, "A Parallel PageRank Algorithm For
 * Undirected Graph") computes the PageRank vector of an undirected graph,
 *
 *     pi* = (1 - c) (I - c P)^-1 p,   P = A D^-1            (Sec. 2.1)
 *
 * by the Chebyshev expansion of f(x) = 1/(1 - c x) applied to P (Eq. 31):
 *
 *     pi_M = c_0/2 p + sum_{k=1..M} c_k T_k(P) p,           (Sec. 4.1)
 *     T_0 p = p,  T_1 p = P p,  T_{k+1} p = 2 P T_k p - T_{k-1} p,
 *
 * followed by a normalisation (Algorithm 1).  The number of rounds M is the
 * smallest one whose rigorous L1 bound is below the caller's tolerance: the
 * tail of the series is ERR_M (Eq. 41) times kappa = sqrt(sum_i d_i) *
 * ||D^-1/2 p||_2, which bounds ||T_k(P) p||_1 for every k.
 *
 * Conventions for every entry point:
 *  - Plain C types only; no exception or C++ type crosses this boundary.
 *  - Every call returns a cpaa_status; nothing aborts the process.
 *    cpaa_last_error() gives a one-line message for the calling thread.
 *  - The caller owns every pointer it passes.  Host arrays may be freed as
 *    soon as a call returns.  Device arrays must stay valid until the work
 *    queued on the caller's stream is complete.
 *  - Graph arrays are CSR with int32 indices: row_ptr[n+1], col_idx[nnz].
 *    Row u lists the neighbours of u in strictly ascending order.  The
 *    matrix is symmetric (undirected graph, Sec. 2.1), and every vertex has
 *    degree >= 1 (d_i > 0, Sec. 2.1).  A self-loop is one entry and counts
 *    once in d_u.  nnz < 2^31.
 *  - Vectors p and pi are FP64, length n.  Batches are B such vectors stored
 *    one after another (column-major n x B).
 *  - A cpaa_graph may be used by one solve at a time; it owns its device
 *    copy of the CSR, its tiling and a reusable workspace.
 *
 * Tests and the Python binding call exactly these symbols.
 */
#ifndef CPAA_H
#define CPAA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CPAA_OK = 0,
    CPAA_EINVAL = 1,     /* bad argument: c outside (0,1), tol <= 0, p < 0, sum p != 1,
                            invalid CSR (see cpaa_graph_create) */
    CPAA_ENOMEM = 2,     /* a device or host allocation failed, or a budget was exceeded */
    CPAA_ENOTCONV = 3,   /* the bound needs more rounds than max_rounds; pi holds the
                            result after max_rounds */
    CPAA_ECUDA = 4,      /* a CUDA runtime call failed (message in cpaa_last_error) */
    CPAA_ETIMEOUT = 5,   /* a wait ran out of time (server) */
    CPAA_EBUSY = 6,      /* no room for the request right now (server) */
    CPAA_ECANCELLED = 7, /* the request was cancelled (server) */
    CPAA_ENOTFOUND = 8   /* unknown ticket or graph id (server) */
} cpaa_status;

/* Number format of the iterate vectors.  F64: FP64 storage and arithmetic.
 * F32: FP32 storage and arithmetic, Kahan-compensated FP32 accumulator.
 * BF16: bfloat16 storage, FP32 arithmetic, Kahan-compensated FP32
 * accumulator.  DF64: double-float -- every value is an unevaluated sum of
 * two FP32 numbers (about 48 significant bits, FP32 exponent range), with
 * error-free FP32 transformations for the arithmetic: FP64-class accuracy on
 * the FP32 pipes of a GPU whose FP64 rate is low.  The coefficients c_k, the
 * stopping rule and every output stay FP64 on all four. */
typedef enum { CPAA_F64 = 0, CPAA_F32 = 1, CPAA_BF16 = 2, CPAA_DF64 = 3 } cpaa_precision;

/* cpaa_graph_create flags */
#define CPAA_GRAPH_DEVICE_INPUT 1u /* row_ptr / col_idx are device pointers */
#define CPAA_GRAPH_VALIDATE 2u     /* accepted and ignored: the row-order and symmetry
                                      checks it once enabled are now the default */
#define CPAA_GRAPH_TRUSTED 4u      /* skip the row-order and symmetry checks (one device
                                      pass over col_idx) for a CSR the caller has already
                                      checked; the column range is checked regardless */
#define CPAA_GRAPH_AUTOTUNE 8u     /* cpaa_graph_create_ex: pick the layout parameters by
                                      timing rounds on candidate layouts (see there) */

/* cpaa_options.flags */
#define CPAA_DEVICE_IO 1u   /* p / pi (P / PI) are device pointers */
#define CPAA_TIME_ROUNDS 2u /* time the M round launches with CUDA events on the solve's
                               stream; the result is cpaa_info.rounds_ms */
#define CPAA_SPARSE_FRONTIER 8u /* early rounds only on the work items that hold a row of the
                                   k-hop ball of p's support (T_k p vanishes outside it,
                                   Sec. 4.1), until that ball covers half the entries or 8
                                   rounds have run; results are the same bits as without it.
                                   cpaa_solve, cpaa_solve_batch and cpaa_server_create (not
                                   with CPAA_SERVER_FUSED); ignored by cpaa_power_solve */
#define CPAA_INTERVAL 16u /* run the series on [cpaa_options.lambda_lo, 1]: the caller
                             certifies that every eigenvalue of P is >= lambda_lo */
#define CPAA_CERTIFY_INTERVAL 32u /* run it on [b, 1] with b the lower bound the graph
                                     certifies by itself (cpaa_graph_spectrum_bound); with
                                     CPAA_INTERVAL too, the larger of b and lambda_lo */
#define CPAA_SERVER_FUSED 4u /* cpaa_server_create: all graphs on one stream, each round of
                                every graph with live queries in one kernel launch over the
                                graphs' work lists, instead of one stream and one launch per
                                graph (results are the same bits either way) */

/* cpaa_options.stop_rule.  The paper runs a fixed M and bounds the truncation
 * by ERR_M = 2 beta^(M+1) / (1 + beta) (Eq. 41), a bound on the neglected
 * mass.  It becomes an L1 bound on pi through the size of the neglected terms
 * T_k p (k > M):
 *   RIGOROUS    ||T_k p||_1 <= kappa = sqrt(sum d) ||D^-1/2 p||_2 for every k
 *               (||T_k(S)||_2 <= 1 for the symmetric S = D^-1/2 A D^-1/2),
 *               so M is fixed before the rounds from ERR_M kappa < tol (plus
 *               the normalisation term of the divide-by-sum form);
 *   POSTERIORI  kappa is replaced by 2 max_{j<=M} ||T_j p||_1, measured by the
 *               rounds' own sums; a vector stops after the first round M that
 *               passes, or at the rigorous M if that comes first.  Not a
 *               proof but an estimate (checked against exact solutions in the
 *               tests).  On power-law graphs a one-seed vector's ||T_j p||_1
 *               climbs to about 0.4 kappa, so it saves a round or two there;
 *               for uniform p, 2 max ||T_j p||_1 exceeds kappa and the rigorous
 *               M stands.  Every round then takes its sums (two small extra
 *               kernels per round). */
typedef enum { CPAA_STOP_RIGOROUS = 0, CPAA_STOP_POSTERIORI = 1 } cpaa_stop_rule;

typedef struct {
    cpaa_precision precision; /* default CPAA_F64 */
    int normalize;            /* 0: pi = pibar / sum(pibar), last line of Algorithm 1 (default);
                                 1: pi = (1 - c) pibar (Sec. 2.1) */
    int fixed_rounds;         /* > 0: run exactly this many rounds (Algorithm 1's M) and
                                 ignore tol; 0: choose M from tol (default) */
    int max_rounds;           /* cap on M; 0 means 2000 */
    unsigned flags;           /* CPAA_DEVICE_IO | CPAA_TIME_ROUNDS | CPAA_SPARSE_FRONTIER |
                                 CPAA_INTERVAL | CPAA_CERTIFY_INTERVAL */
    void *stream;             /* cudaStream_t to run on; NULL = legacy default stream */
    double *history;          /* optional host array [2*(M+1)]: sum T_k and sum |T_k|
                                 for k = 0..M (the mass view of Sec. 4.1); cpaa_solve only */
    int batch_width;          /* cpaa_solve_batch: vectors per tile, 1/2/4/8/16, or 0 (default):
                                 the first batch of at least 16 columns of a precision on a
                                 graph times a few rounds at every width on its own columns
                                 and keeps the fastest per column for that graph */
    cpaa_stop_rule stop_rule; /* default CPAA_STOP_RIGOROUS; cpaa_solve and cpaa_solve_batch */
    double lambda_lo;         /* with CPAA_INTERVAL: the lower end of an interval [lambda_lo, 1]
                                 that holds every eigenvalue of P (they are real and >= -1,
                                 Lemma 2); default -1, read only under that flag.  The series
                                 of Sec. 2.2 then runs on the narrower interval: the recurrence
                                 on Q = (P - mid I) / half (mid, half the interval's centre and
                                 half-width) with coefficients c_k(chat) / (1 - c mid),
                                 chat = c half / (1 - c mid) < c, so it converges faster and
                                 fewer rounds reach tol.  Must lie in [-1, 1).  A value above
                                 the true smallest eigenvalue gives wrong results: it must be
                                 a proven bound.  cpaa_solve and cpaa_solve_batch; the server
                                 rejects both interval flags and the power method ignores them */
} cpaa_options;

typedef struct {
    int rounds;       /* M that was run (accumulated terms c_1 .. c_M) */
    double bound;     /* L1 bound on ||pi - pi*||_1 after M rounds by the stop rule that
                         ended the solve: rigorous, or the a-posteriori estimate */
    double kappa;     /* sqrt(sum d) ||D^-1/2 p||_2 */
    double mass;      /* sum_u T_M[u]; equals sum p up to rounding (Sec. 4.1) */
    double l1;        /* sum_u |T_M[u]| */
    double sum_pibar; /* sum_u pibar[u] before normalisation */
    double rounds_ms; /* device time of the M round launches (CPAA_TIME_ROUNDS), else 0 */
    double lambda_lo; /* lower end of the interval the series ran on (-1: Algorithm 1's) */
} cpaa_info;

typedef struct cpaa_graph cpaa_graph;

/* Fill *opt with the defaults listed above. */
void cpaa_options_init(cpaa_options *opt);

/* Upload an undirected graph (Sec. 2.1: A symmetric, d_i > 0) and build the
 * degree vectors and the row tiling the step kernels walk.
 *   n        vertices, 1 <= n < 2^31
 *   nnz      CSR entries, row_ptr[n]; 0 < nnz < 2^31
 *   row_ptr  int32[n+1], host or device (CPAA_GRAPH_DEVICE_INPUT)
 *   col_idx  int32[nnz], same memory space as row_ptr
 *   flags    CPAA_GRAPH_DEVICE_INPUT | CPAA_GRAPH_TRUSTED
 *   out      receives the handle; release with cpaa_graph_destroy
 * Always checked: row_ptr[0] = 0, row_ptr non-decreasing, row_ptr[n] = nnz,
 * every degree >= 1 (on the host), and 0 <= col_idx < n (on the device, in
 * the relabelling pass; an out-of-range id is never used as an index).
 * Unless CPAA_GRAPH_TRUSTED is given, also: strictly ascending rows (no
 * duplicate entries) and A symmetric (the remark closing Sec. 3: Eq. 31 needs
 * the real spectrum that an undirected graph gives).  Violations return
 * CPAA_EINVAL, with the counts in cpaa_last_error, and no handle.  Runs on
 * the current CUDA device. */
cpaa_status cpaa_graph_create(int64_t n, int64_t nnz, const int32_t *row_ptr,
                              const int32_t *col_idx, unsigned flags, cpaa_graph **out);

/* Release the graph and its workspace.  NULL is accepted. */
cpaa_status cpaa_graph_destroy(cpaa_graph *g);

/* Size of the graph and the device bytes it holds (CSR, degrees, tiling and
 * workspace).  Any output pointer may be NULL. */
cpaa_status cpaa_graph_info(const cpaa_graph *g, int64_t *n, int64_t *nnz,
                            int64_t *device_bytes, int64_t *num_tiles);

/* How cpaa_graph_create laid the graph out for the round kernels (no paper
 * counterpart: this is the GPU layout).  Rows above hub_degree are hub rows,
 * kept as CSR and cut into tiles of hub_tile entries, one CTA per tile; the
 * other rows, sorted by degree within windows of sort_window rows, form SELL
 * chunks of 32 rows (sell_entries counts their stored entries with padding),
 * of which long_chunks, those whose longest row exceeds long_chunk entries
 * (or 65532, whichever is smaller: a warp's rows read a 2-byte degree),
 * get a CTA and the rest a warp.  tuned = 1 when CPAA_GRAPH_AUTOTUNE picked
 * the parameters after timing tune_candidates layouts. */
typedef struct {
    int64_t hub_rows, hub_entries, hub_tiles;
    int64_t chunks, long_chunks, sell_entries;
    int hub_degree, hub_tile;
    int long_chunk, sort_window;
    int tuned, tune_candidates;
} cpaa_layout;

cpaa_status cpaa_graph_layout(const cpaa_graph *g, cpaa_layout *out);

/* Layout parameters for cpaa_graph_create_ex (no paper counterpart).  A field
 * left at 0 takes its default: hub_degree min(4096, max(64, nnz / 4096)),
 * hub_tile twice the hub degree within [512, 8192], long_chunk 32 (8 below
 * 2^22 entries), sort_window 1024.  Limits: hub_degree >= 32; hub_tile a
 * multiple of 4 in [256, 2^20]; sort_window a multiple of 32 up to 2^20;
 * otherwise CPAA_EINVAL.  tune_precision is the number format the autotuner
 * times rounds in (a cpaa_precision; 0 = CPAA_F64). */
typedef struct {
    int hub_degree, hub_tile, long_chunk, sort_window;
    int tune_precision;
} cpaa_layout_params;

/* cpaa_graph_create with explicit layout parameters (params NULL: all
 * defaults).  With CPAA_GRAPH_AUTOTUNE in flags the parameters are a starting
 * point: the call builds candidate layouts around them (sort window, then hub
 * threshold, hub tile and long-chunk threshold, a coordinate search of at most
 * 13 layouts), times a few single-vector rounds of uniform p on each in
 * tune_precision (CUDA events), and returns the graph with the fastest; the
 * pick is cached for the rest of the process by device, size and degree
 * histogram, so a second such call on a like graph builds one layout.
 * Results of every layout agree to rounding (the sums run in another order).
 * Other arguments, checks and errors as cpaa_graph_create. */
cpaa_status cpaa_graph_create_ex(int64_t n, int64_t nnz, const int32_t *row_ptr,
                                 const int32_t *col_idx, unsigned flags,
                                 const cpaa_layout_params *params, cpaa_graph **out);

/* Personalised PageRank of one vector (Sec. 2.1, Algorithm 1).
 *   p    FP64[n], p >= 0, |sum p - 1| <= 1e-9
 *   c    damping factor, 0 < c < 1
 *   tol  L1 tolerance on ||pi - pi*||_1 (> 0; ignored with fixed_rounds)
 *   pi   FP64[n] output
 *   opt  NULL for defaults
 *   info NULL or receives the run's figures
 * p and pi are host pointers unless opt->flags has CPAA_DEVICE_IO.  With host
 * pointers the call returns once pi is written; with device pointers it
 * returns once the work is queued behind one short synchronisation (the
 * rounds M depend on kappa, which is reduced on the device). */
cpaa_status cpaa_solve(cpaa_graph *g, const double *p, double c, double tol, double *pi,
                       const cpaa_options *opt, cpaa_info *info);

/* The paper's comparison baseline on the same device layout and kernels: the
 * power method x <- c P x + (1 - c) p from x = p (the SPI of Sec. 5.1, also its
 * ground truth).  It runs T rounds, the smallest with 2 c^T < tol (since
 * ||x_T - pi*||_1 <= c^T ||p - pi*||_1 <= 2 c^T), or opt->fixed_rounds.
 * Arguments, info (bound = 2 c^T) and errors as cpaa_solve; CPAA_F64, CPAA_F32
 * or CPAA_DF64.  normalize = 1 returns x_T as it is (it sums to 1 up to
 * rounding); normalize = 0 divides by its sum. */
cpaa_status cpaa_power_solve(cpaa_graph *g, const double *p, double c, double tol, double *pi,
                             const cpaa_options *opt, cpaa_info *info);

/* B personalised vectors at once (the batched form: the graph is read once
 * per step for a whole tile of vectors).  Column b of P (P + b*n) is solved
 * with damping c[b] and written to PI + b*n; info, if not NULL, has B
 * entries.  Each column gets the rounds its own bound asks for; a column's
 * result does not depend on the other columns. */
cpaa_status cpaa_solve_batch(cpaa_graph *g, int B, const double *P, const double *c,
                             double tol, double *PI, const cpaa_options *opt,
                             cpaa_info *info);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over resident graphs.
 *
 * Queries are personalised PageRank vectors with a few seed vertices, each
 * with its own damping c and tolerance (Sec. 2.1: p uniform over the seeds,
 * or weighted).  Every added graph gets a fixed number of column slots whose
 * device memory is reserved from the server's budget when the graph is added;
 * a query waits in its graph's queue until a slot is free, then joins the
 * graph's running tile before the next round, while the other columns of the
 * tile keep going (each column has its own round counter, coefficients and
 * stopping round).  A query takes the graph's lowest free slot, and each
 * round computes only the narrowest power-of-two prefix of the slots that
 * holds every running query (the tile's vectors are re-laid out at that width
 * when it changes), so a lone query costs a single-vector round and a full
 * graph one round of all its slots.  Each graph runs on its own CUDA stream, so the work of
 * different graphs overlaps on the device (or, with CPAA_SERVER_FUSED, one
 * launch per round covers every graph with live queries).  A query's result
 * does not depend on what else is running: every column's arithmetic is the
 * same, in the same order, whatever the other columns hold.
 * ------------------------------------------------------------------------ */
typedef struct cpaa_server cpaa_server;

/* Most seed vertices one query may name. */
#define CPAA_SERVER_MAX_SEEDS 64

typedef struct {
    uint64_t submitted, completed, cancelled, failed;
    int64_t pending;      /* queued, not yet in a slot */
    int64_t running;      /* in a slot */
    int64_t slots;        /* total slots over all graphs */
    int64_t device_bytes; /* reserved from the budget */
    double p50_us, p99_us, mean_us; /* submit -> result ready, completed queries */
    double admit_p50_us;  /* submit -> slot */
    uint64_t rounds;        /* rounds launched, over all graphs */
    uint64_t round_columns; /* sum over those rounds of the tile width (columns computed) */
    uint64_t relayouts;     /* tile width changes */
} cpaa_server_stats;

/* Create a server.  device_mem_budget bounds the device memory of all slots;
 * opt (NULL for defaults) sets the precision (any of the four; default for
 * serving: CPAA_F32), normalize, max_rounds and
 * stop_rule; of its flags only CPAA_SERVER_FUSED and CPAA_SPARSE_FRONTIER are read
 * (the frontier applies to graphs of at least 2^22 entries whose tile starts
 * from empty: their first rounds skip the work items outside the queries'
 * k-hop balls until a query joins the running ones), and its stream is
 * ignored.  Starts two host threads (scheduler, completion). */
cpaa_status cpaa_server_create(size_t device_mem_budget, const cpaa_options *opt,
                               cpaa_server **out);

/* Make a graph resident in the server with up to max_slots (1..16, rounded
 * down to a power of two; 0 = 16) concurrent queries, as many as the remaining
 * budget allows.  CPAA_ENOMEM if not even one slot fits.  The graph must
 * outlive the server and must not be used by other calls while the server
 * runs.  *graph_id receives the id for cpaa_server_submit. */
cpaa_status cpaa_server_add_graph(cpaa_server *s, cpaa_graph *g, int max_slots, int *graph_id);

/* Queue a query: seeds[nseeds] (distinct vertex ids, 1 <= nseeds <=
 * CPAA_SERVER_MAX_SEEDS), weights[nseeds] (>= 0, summing to 1; NULL for
 * uniform 1/nseeds), damping c in (0,1), L1 tolerance tol > 0.  Returns at
 * once with a ticket.  CPAA_EBUSY if the graph's queue is full. */
cpaa_status cpaa_server_submit(cpaa_server *s, int graph_id, int nseeds, const int32_t *seeds,
                               const double *weights, double c, double tol, uint64_t *ticket);

/* Wait up to timeout_us (< 0: forever) for a query.  A finished query's vector
 * waits in its slot's device memory (holding the slot) until this call copies
 * it to pi -- n doubles in the caller's vertex order, host or device memory,
 * or NULL to discard it -- fills info (may be NULL; rounds and bound are those
 * of the stop rule that ended the query; mass, l1 and sum_pibar are NaN: they
 * are not reported when serving), frees the slot and releases the ticket.  CPAA_ETIMEOUT leaves the query in place; CPAA_ECANCELLED releases a
 * cancelled query; CPAA_ENOTFOUND names no query. */
cpaa_status cpaa_server_wait(cpaa_server *s, uint64_t ticket, double *pi, cpaa_info *info,
                             int64_t timeout_us);

/* Cancel a query: a queued or running one leaves its slot at the next round, a
 * finished one's uncollected vector is discarded. */
cpaa_status cpaa_server_cancel(cpaa_server *s, uint64_t ticket);

/* Counters and latency percentiles so far. */
cpaa_status cpaa_server_get_stats(cpaa_server *s, cpaa_server_stats *out);

/* Stop the threads (running queries are cancelled) and free the slots. */
cpaa_status cpaa_server_destroy(cpaa_server *s);

/* Largest n that cpaa_solve_fixed_noalloc accepts.  That call keeps two FP64
 * iterate vectors and an FP64 accumulator (24 bytes per vertex) plus a small
 * reduction area in a fixed 32 MiB scratch array per GPU. */
#define CPAA_NOALLOC_MAX_N 1300000

/* Solve without allocating any memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory
 * themselves -- code running inside an application whose allocator owns the
 * device (a framework's caching allocator or a fixed arena), a process held to
 * a strict memory budget, or a loop that cannot afford the device-wide
 * synchronisation cudaMalloc / cudaFree can cause.  It calls no allocation
 * routine; all its intermediate vectors live in one 32 MiB device array that
 * the library reserves on every GPU that loads it, for the life of the process.
 *   n, nnz, row_ptr, col_idx  the graph as for cpaa_graph_create, in DEVICE
 *                             memory; 1 <= n <= CPAA_NOALLOC_MAX_N
 *   p                         FP64[n] in device memory, p >= 0, sum 1 (not checked)
 *   c                         damping factor in (0, 1)
 *   rounds                    number of recurrence rounds (0..2000);
 *                             cpaa_rounds_needed gives it for a tolerance
 *   normalize                 as in cpaa_options
 *   pi                        FP64[n] output in device memory
 *   stream                    cudaStream_t, NULL = legacy default stream
 * Arithmetic is FP64 and matches cpaa_solve with fixed_rounds = rounds to
 * rounding.  Every call blocks: it reads back an error counter and returns
 * only after the stream has finished its work, so it must never be called on
 * a stream that is being captured into a CUDA graph.  It returns CPAA_EINVAL
 * if n is beyond CPAA_NOALLOC_MAX_N or an argument is out of range, and also
 * if the CSR has a column outside [0, n) or a row of degree <= 0, whatever
 * `rounds` is (such entries are skipped, never read out of bounds).  A call on
 * a device whose scratch address is not yet known looks it up first (a failed
 * lookup is retried by the next call).  All calls share that array and it
 * keeps the previous call's contents; calls that overlap on the GPU race, so
 * serialise them. */
cpaa_status cpaa_solve_fixed_noalloc(int64_t n, int64_t nnz, const int32_t *row_ptr,
                                     const int32_t *col_idx, const double *p, double c,
                                     int rounds, int normalize, double *pi, void *stream);

/* The stopping rule on its own: the smallest M in [1, max_rounds] with
 * bound(M) < tol, or -1.  normalize as in cpaa_options; bound as in
 * cpaa_info.bound (Eq. 41 times kappa, plus the normalisation term). */
int cpaa_rounds_needed(double c, double tol, double kappa, int normalize, int max_rounds);

/* The bound itself for a given M. */
double cpaa_l1_bound(double c, int M, double kappa, int normalize);

/* The same two for the series on [lambda_lo, 1] (cpaa_options.lambda_lo): Eq. 41's
 * ERR_M becomes the mass the truncated interval series leaves out,
 * (1 - c) sum_{k>M} c_k, which kappa turns into an L1 bound as before (Q is
 * similar to a symmetric matrix whose spectrum lies in [-1, 1]).  lambda_lo =
 * -1 gives the functions above.  -1 (rounds) or NaN (bound) for arguments out
 * of range. */
int cpaa_rounds_needed_interval(double c, double lambda_lo, double tol, double kappa, int normalize,
                                int max_rounds);
double cpaa_l1_bound_interval(double c, double lambda_lo, int M, double kappa, int normalize);

/* The lower bound on P's spectrum that the graph certifies by itself: with a
 * self-loop on every vertex, D' + A' (the loop-free degree and adjacency
 * matrices) is positive semidefinite, so A + D >= 2I and every eigenvalue of
 * D^-1/2 A D^-1/2 is at least -1 + 2 / d_max; otherwise -1 (Lemma 2's).  No
 * paper counterpart: the paper's series is on [-1, 1]. */
cpaa_status cpaa_graph_spectrum_bound(const cpaa_graph *g, double *lambda_lo);

/* Human-readable name of a status. */
const char *cpaa_status_string(cpaa_status s);

/* Message of the last failing call on this thread ("" if none). */
const char *cpaa_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CPAA_H */
