// internal.h -- shared definitions of the CPAA library (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "cpaa.h"

namespace cpaa {

// ---------------------------------------------------------------------------
// Layout of the graph on the device.
//
// Vertices are relabelled once, at cpaa_graph_create:
//   new ids [0, n_hub)  hub rows (degree > hub_degree(nnz)), by decreasing degree;
//   new ids [n_hub, n)  heavy rows (degree at least kHeavyMin and kHeavyFactor times the mean)
//                       by decreasing degree, then every other row in the
//                       original order; cut into windows of kSortWindow rows,
//                       each window sorted by decreasing degree.
// Every per-vertex vector (degrees, iterates, accumulator) is stored in the new
// order; the solve gathers p through the permutation and scatters pi back.
// Every row's entries are the relabelled graph's CSR row: new column ids,
// ascending (so a row starts with its hub and heavy neighbours).
//
// Non-hub rows are held as SELL-C-sigma (sliced ELLPACK, C = kChunkRows = 32,
// sigma = kSortWindow): chunk c holds new rows n_hub + 32c .. + 31, padded to
// the chunk's longest row rounded up to a multiple of kSellVec, column-major
// in groups of kSellVec entries per lane (entry i of lane l at
// chunk_off[c] + 128 (i / 4) + 4 l + i % 4, so a warp reads 512 contiguous
// bytes per load); padding entries hold the sentinel column n, whose iterate
// value is kept at zero.  One warp owns one chunk, one lane one row.  The
// round kernel reads each lane's first L entries only, L the chunk's longest
// row (kept in the chunk's descriptor): a last, partial group gives its first
// L mod kSellVec entries, so no sentinel is gathered past the longest row.
// Windows are multiples of 32 rows, so a chunk never straddles two windows
// and its first row is its longest.
//
// The hub threshold is kHubDegree on large graphs.  A small graph lowers it
// (nnz / 4096, at least kMinHubDegree): its round is short, and a SELL chunk
// whose first rows are long would otherwise set the round's length by one
// lane's serial gathers (and carry the padding of its shorter rows).  A hub
// tile holds twice the hub threshold, within [kMinHubTile, kMaxHubTile]
// entries: long tiles on large graphs (fewer barriers and tickets per entry),
// short ones on small graphs (more CTAs on a row).
//
// Hub rows stay CSR (relabelled columns, ascending).  Their entries are cut into tiles;
// one CTA sums one tile, and the CTA that takes the last ticket of a row adds
// the tile partials in tile order and writes the row (an atomic counter, no
// waiting).  Hub tile encoding (int4):
//   {row, tile, slot, hub + 1}   slot = partial-sum index of tile 0 of the row
//
// Defaults of the thresholds: timed on the 2^24-vertex Chung-Lu graph (single
// FP32 vector) against hub thresholds of 1024 to 16384, tiles of 1024 to 16384
// entries and long-chunk thresholds of 32 to 128, and on the 10^4-vertex one
// (FP64), where graphs below 2^22 entries take long chunks above 8 entries
// and hub tiles down to 512 entries: there a round is a chain of latencies.
// Every threshold and the sort window are per-graph parameters
// (cpaa_layout_params); CPAA_GRAPH_AUTOTUNE picks them by timing rounds.
// ---------------------------------------------------------------------------
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunkRows = 32;
constexpr int kSellVec = 4;     // a lane's SELL entries are stored in groups of 4 (one 16-byte load)
#ifndef CPAA_SORT_WINDOW
#define CPAA_SORT_WINDOW 1024
#endif
constexpr int kSortWindow = CPAA_SORT_WINDOW;  // sigma of SELL-C-sigma (a multiple of 32)
#ifndef CPAA_HEAVY_FACTOR
#define CPAA_HEAVY_FACTOR 2
#endif
#ifndef CPAA_HEAVY_MIN
#define CPAA_HEAVY_MIN 64
#endif
constexpr int kHeavyFactor = CPAA_HEAVY_FACTOR;  // heavy rows: degree >= this times the mean
constexpr int kHeavyMin = CPAA_HEAVY_MIN;        // ... and >= this
// Tuning constants (compile-time; the defaults were picked by timing the
// round on the 2^24-vertex Chung-Lu graph).
#ifndef CPAA_HUB_DEGREE
#define CPAA_HUB_DEGREE 4096
#endif
#ifndef CPAA_MAX_HUB_TILE
#define CPAA_MAX_HUB_TILE 8192
#endif
#ifndef CPAA_LONG_CHUNK
#define CPAA_LONG_CHUNK 32
#endif
constexpr int kHubDegree = CPAA_HUB_DEGREE;       // hub rows: degree above this (the cap)
#ifndef CPAA_MIN_HUB_DEGREE
#define CPAA_MIN_HUB_DEGREE 64
#endif
#ifndef CPAA_MIN_HUB_TILE
#define CPAA_MIN_HUB_TILE 512
#endif
#ifndef CPAA_SMALL_LONG_CHUNK
#define CPAA_SMALL_LONG_CHUNK 8
#endif
constexpr int kMinHubDegree = CPAA_MIN_HUB_DEGREE;
constexpr int kMaxHubTile = CPAA_MAX_HUB_TILE;    // entries of a hub tile (the cap)
constexpr int kMinHubTile = CPAA_MIN_HUB_TILE;
constexpr int kSmallLongChunk = CPAA_SMALL_LONG_CHUNK;  // long-chunk threshold of small graphs
constexpr int kLongChunk = CPAA_LONG_CHUNK;       // SELL chunks longer than this get a whole CTA
constexpr int kSumBlocks = 256; // CTAs of the first level of the per-round item sums
constexpr int kDefaultMaxRounds = 2000;

constexpr int kPrepBlocks = 1024;  // CTAs of the fixed-order reductions
constexpr int kMaxWidth = 16;      // widest tile of vectors a round kernel takes
// Longest row a short (warp) SELL chunk may hold: its rows read their degree
// as a 2-byte word, so chunks with longer rows are long (CTA) chunks whatever
// the long-chunk threshold.
constexpr int kMaxShortRow = 65532;

// Layout parameters of a graph (cpaa_layout_params with every default
// resolved): hub rows have degree above hub_degree and are cut into tiles of
// hub_tile entries; SELL chunks whose longest row exceeds long_chunk get a
// CTA; rows are sorted by degree within windows of sort_window rows.
struct LayoutParams {
    int hub_degree = 0;
    int hub_tile = 0;
    int long_chunk = 0;
    int sort_window = 0;
};

// A double-float value: hi + lo, |lo| <= ulp(hi) / 2 (CPAA_DF64).  The
// arithmetic is in device_common.cuh.
struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ explicit df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
};

// Sparse-frontier state (CPAA_SPARSE_FRONTIER).  T_k p is zero outside the
// k-hop ball of p's support (Sec. 4.1: T_{k+1} = 2 P T_k - T_{k-1} adds one hop
// per round), so early rounds need only the work items (hub tiles, SELL
// chunks) that hold a row of that ball.  Bitmaps over the rows, one bit per
// row in the layout's order: words [0, hub_words) for the hub rows, then one
// 32-bit word per SELL chunk (bit l: the chunk's row l).
struct Frontier {
    unsigned *cur = nullptr;   // rows that may be nonzero in a live column (cumulative)
    unsigned *ring = nullptr;  // rows added by the last update: expanded next
    unsigned *add = nullptr;   // neighbours marked by the last expansion
    int *full = nullptr;       // sticky: 1 once rounds run over every item
    unsigned long long *entries = nullptr;  // [2] stored entries of the items cur covers, by update parity
    int64_t words = 0;
    int hub_words = 0;
};
// Rounds that may run on the frontier (later ones always run on every item),
// and the covered share of the entries beyond which rounds run on every item.
constexpr int kFrontierRounds = 8;
constexpr int kFrontierLimitDiv = 2;  // limit = nnz / kFrontierLimitDiv stored entries

// Workspace of the solves, grown on demand and reused (one solve per graph at
// a time).  Vectors of a tile of W columns are row-major [rows x W].
struct Workspace {
    void *y0 = nullptr;        // iterates y = D^-1 T, [(n+1) x W] (row n: zero sentinel)
    void *y1 = nullptr;
    size_t vec_bytes = 0;
    void *rho = nullptr;       // accumulator D^-1 pibar, [n x W]
    void *comp = nullptr;      // Kahan compensation (FP32 paths), [n x W]
    size_t rho_bytes = 0;
    double *red = nullptr;     // per-round sums [(M+1)][2][W]: sum T, sum |T| per column
    size_t red_bytes = 0;
    double *ipart = nullptr;   // item partial sums [(n_hub + num_chunks)][2][W]
    size_t ipart_bytes = 0;
    double *ipart2 = nullptr;  // first-level sums [kSumBlocks][2][W]
    // a-posteriori stopping rule (CPAA_STOP_POSTERIORI): per column
    double *maxl1 = nullptr;   // running max_j ||T_j p||_1 [kMaxWidth]
    unsigned *stop = nullptr;  // stopped columns
    int *stop_round = nullptr; // [kMaxWidth]
    void *long_part = nullptr; // hub tile partials [num_hub_tiles x W]
    size_t long_part_bytes = 0;
    double *part = nullptr;    // per-CTA partials of the fixed-order reductions
    double *sums = nullptr;    // reduced scalars (device)
    double *h_sums = nullptr;  // pinned host copy of sums
    double *io = nullptr;      // device staging of host p / pi
    size_t io_bytes = 0;
    // Round sequences captured as CUDA graphs (solve.cu), keyed by every
    // value the launches take; replayed by later solves with the same key.
    struct RoundGraph {
        std::vector<uint64_t> key;
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<RoundGraph> round_graphs;
    cudaStream_t capture = nullptr;  // private stream the captures run on
    cudaEvent_t tev[2] = {nullptr, nullptr};  // around the rounds (CPAA_TIME_ROUNDS)
    Frontier fr;                     // CPAA_SPARSE_FRONTIER solves (allocated on first use)
    // the interval series' factor ia * 2 / d by degree (tab_n entries of the
    // solve's arithmetic type; filled per solve on [lambda_lo, 1])
    void *ivtab = nullptr;
};

// One tile of up to kMaxWidth vectors for run_tile (solve.cu).
struct TileJob {
    int width = 1;
    int precision = CPAA_F64;
    int normalize = 0;
    const double *p[kMaxWidth] = {};  // device input columns (caller's vertex order)
    double *pi[kMaxWidth] = {};       // device output columns
    double c[kMaxWidth] = {};
    double c0half[kMaxWidth] = {};   // power method: 1 - c (the accumulator slot holds q)
    int rounds[kMaxWidth] = {};
    int power = 0;                    // 1: power-method rounds instead of Chebyshev ones
    int frontier = 0;                 // 1: early rounds on the sparse frontier (CPAA_SPARSE_FRONTIER)
    double lambda_lo = -1.0;          // the series' interval [lambda_lo, 1] (-1: Algorithm 1's)
    int posteriori = 0;               // 1: columns may stop early by the a-posteriori rule
    double tol = 0;                   // its tolerance
    double p_l1[kMaxWidth] = {};      // ||p||_1 = ||T_0 p||_1 of each column (that rule's start)
};

// The a-posteriori stopping rule for one round (solve.cu): after round k,
// column b stops when ERR_k(c_b) * 2 max_{j<=k} ||T_j p||_1 (plus the
// normalisation term of the divide-by-sum form) falls below tol.
struct StopArgs {
    unsigned decide = 0;            // columns that test the rule this round
    int k[kMaxWidth] = {};          // each column's round number
    double err[kMaxWidth] = {};     // ERR_k of each column at that round (Eq. 41)
    double tol[kMaxWidth] = {};     // each column's tolerance
    int normalize = 0;
    double *maxl1 = nullptr;        // [W] running max of ||T_j p||_1, j <= k
    unsigned *stop = nullptr;       // stopped columns (bit mask)
    int *stop_round = nullptr;      // [W] the round a column stopped after
};

}  // namespace cpaa

struct cpaa_graph {
    int64_t n = 0;
    int64_t nnz = 0;
    int device = 0;
    int32_t *perm = nullptr;         // new id -> original id [n]
    // hub rows (CSR, relabelled)
    int n_hub = 0;
    int64_t hub_nnz = 0;
    int32_t *hub_row_ptr = nullptr;  // [n_hub + 1]
    int32_t *hub_col = nullptr;      // [hub_nnz + 4]
    int4 *hub_tiles = nullptr;
    int num_hub_tiles = 0;
    int *long_cnt = nullptr;         // per hub row ticket counter [n_hub], kept at zero
    // other rows (SELL-C-sigma, relabelled)
    int num_chunks = 0;
    int64_t sell_entries = 0;        // including padding
    int32_t *sell_col = nullptr;     // [sell_entries]
    int64_t *chunk_off = nullptr;    // [num_chunks]
    int32_t *chunk_len = nullptr;    // [num_chunks]
    int32_t *chunk_order = nullptr;  // chunk ids, longest first
    int4 *chunk_desc = nullptr;      // [num_chunks] in chunk_order: {chunk, offset / 128, length, longest row}
    int hub_degree = cpaa::kHubDegree;  // rows above this degree are hub rows
    int hub_tile = cpaa::kMaxHubTile;   // entries of a hub tile
    int num_long_chunks = 0;         // leading chunk_order entries longer than lp.long_chunk
    cpaa::LayoutParams lp;           // the layout's parameters (hub_degree, hub_tile as above)
    int loops_all = 0;               // 1: every vertex has a self-loop
    int dmax = 0;                    // largest degree
    int tuned = 0;                   // 1: lp picked by timing candidates (CPAA_GRAPH_AUTOTUNE)
    int tune_candidates = 0;         // layouts timed to pick it
    // per-vertex, new order
    double *deg64 = nullptr;         // d_u
    double *inv_deg64 = nullptr;     // 1 / d_u
    double *inv2_deg64 = nullptr;    // 2 / d_u (the recurrence's factor)
    cpaa::df *deg_df = nullptr;      // d_u, 1 / d_u and 2 / d_u as double-floats (CPAA_DF64)
    cpaa::df *inv_deg_df = nullptr;
    cpaa::df *inv2_deg_df = nullptr;
    float *deg32 = nullptr;
    float *inv_deg32 = nullptr;
    float *inv2_deg32 = nullptr;
    // the same three values by degree d in [0, tab_n), rows of tab_n entries:
    // d, 1 / d, 2 / d (entry 0 unused).  A short SELL chunk's rows hold at
    // most min(long_chunk, kMaxShortRow, hub_degree, d_max) = tab_n - 1
    // entries, so the round kernel reads their degree as a 2-byte word
    // (deg16, every vertex: min(d, 65535)) and looks the factors up here
    // instead of reading an 8-byte one
    uint16_t *deg16 = nullptr;
    double *tab64 = nullptr;
    cpaa::df *tab_df = nullptr;
    float *tab32 = nullptr;
    int tab_n = 0;
    int64_t device_bytes = 0;
    int tuned_width[4] = {0, 0, 0, 0};  // batch tile width picked by the autotuner, per precision
    cpaa::Workspace ws;
};

namespace cpaa {

// Thread-local error message plus status.
cpaa_status fail(cpaa_status s, const std::string &msg);
cpaa_status cuda_fail(cudaError_t e, const char *what);
void clear_error();

#define CPAA_CUDA(call)                                        \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cpaa::cuda_fail(e_, #call); \
    } while (0)

// Device allocation tracked in g->device_bytes.
cpaa_status dev_alloc(cpaa_graph *g, void **p, size_t bytes);
void dev_free(cpaa_graph *g, void **p, size_t bytes);

// ERR_M = 2 beta^(M+1) / (1 + beta) (Eq. 41), the expression cpaa_l1_bound uses.
double err_bound(double c, int M);

// Host-side coefficient table c_0..c_M (Sec. 2.2, Proposition 1).
void cheb_coeffs(double c, int M, std::vector<double> &ck);

// The series on [lo, 1] (cpaa_options.lambda_lo; status.cpp): centre, half-width,
// the reduced damping chat and the coefficient scale 1 / (1 - c mid).
struct IntervalMap {
    double mid, half, chat, scale;
};
IntervalMap interval_map(double c, double lo);
void cheb_coeffs_on(double c, double lo, int M, std::vector<double> &ck);  // lo = -1: cheb_coeffs
double err_bound_on(double c, double lo, int M);                           // lo = -1: err_bound
// The graph's own certified lower end (-1 + 2 / d_max with a loop on every
// vertex, else -1; graph.cu), and the interval a solve runs on (solve.cu).
double graph_lambda_lo(const cpaa_graph *g);
cpaa_status resolve_interval(const cpaa_graph *g, const cpaa_options &opt, double *lo);

// Round launcher (step.cu): one round for a tile of `width` vectors.
struct StepLaunch {
    const cpaa_graph *g = nullptr;
    int precision = CPAA_F64;
    int width = 1;                  // 1, 2, 4, 8 or 16
    const void *y_src = nullptr;    // gathered iterates y_{k-1}, [(n+1) x width]
    void *y_io = nullptr;           // in: y_{k-2} (k >= 2); out: y_k
    void *rho = nullptr;            // [n x width]
    void *comp = nullptr;           // [n x width]
    void *long_part = nullptr;      // hub tile partials [num_hub_tiles x width]
    double *ipart = nullptr;        // item partial sums (reducing rounds)
    double *ipart2 = nullptr;       // first-level sums [kSumBlocks][2][width]
    double *red = nullptr;          // this round's sums [2][width]
    const unsigned *stop = nullptr; // stopped columns (a-posteriori rule), or NULL
    StopArgs sa;                    // the rule's test after this round (sa.decide == 0: none)
    double ck[kMaxWidth] = {};
    // Deferred accumulation: a column's term c_k y_k may be added one round
    // late, from the stored y_k, together with c_{k+1} y_{k+1}; the
    // accumulator then takes the same fused operations in the same order, so
    // the result is the same bits, and rounds with no term to add neither read
    // nor write it.  pend: columns whose last round's term is added now (with
    // ck_prev); defer: columns whose term this round is left for the next.
    double ck_prev[kMaxWidth] = {};
    unsigned pend = 0;
    unsigned defer = 0;
    const void *ivtab = nullptr;    // the interval series' factor table (Workspace::ivtab)
    unsigned active = 0;            // columns that still accumulate
    unsigned reduce = 0;            // nonzero: take this round's sums
    unsigned first = 0;             // columns in their first round (k == 1)
    int power = 0;                  // 1: power-method round (ck[b] = c, rho holds q = (1-c) p / d)
    int interval = 0;               // 1: the recurrence on Q = (P - mid I) / half
    double ia = 1.0, mb = 0.0;      // its 1 / half and -2 mid / half
    int *long_cnt = nullptr;        // hub ticket counters [n_hub], all zero; NULL = the graph's own
    // sparse frontier (NULL: every item): items whose rows are all outside
    // front are skipped, unless *front_full or *front_entries > front_limit
    const unsigned *front = nullptr;
    int *front_full = nullptr;
    const unsigned long long *front_entries = nullptr;
    unsigned long long front_limit = 0;
    int front_hub_words = 0;
    cudaStream_t stream = nullptr;
};
void prepare_step(int precision, int width, bool interval = false);
// The series on [lambda_lo, 1] (step_interval.cu; launch_step forwards there
// when StepLaunch::interval is set).
void prepare_step_interval(int precision, int width);
cudaError_t launch_step_interval(const StepLaunch &s);
// The interval series' factor table ia 2 / d by degree, in precision's
// arithmetic type, into out (g->tab_n entries; step_interval.cu).
cudaError_t launch_ivtab(const cpaa_graph *g, int precision, double ia, void *out, cudaStream_t st);
// The deferred-accumulation masks of round k for columns with rounds[b]
// rounds and coefficients ck[b] (solve.cu).
void defer_terms(int k, const int *rounds, int W, const std::vector<std::vector<double>> &ck, StepLaunch &sl);
// Whether the round kernel form for this precision and width takes deferred
// terms (step_impl.cuh, deferred_form): the single-vector FP32, BF16 and DF64
// forms.
inline bool defer_supported(int precision, int width) { return width == 1 && precision != CPAA_F64; }

// Sparse-frontier pieces (frontier.cu).  ensure_frontier allocates f for g
// (frontier_bytes of device memory, counted in track's device_bytes);
// frontier_reset clears it; frontier_mark_nonzero marks the rows where any of
// the `width` columns of y0 is nonzero (and zeroes those rows of y1, the other
// iterate buffer); frontier_mark_rows marks up to kMaxFrontierSeeds given rows;
// frontier_expand adds the neighbours of the last ring and counts the entries
// covered (update parity `parity`); frontier_launch fills a round's fields.
constexpr int kMaxFrontierSeeds = 64;
size_t frontier_bytes(const cpaa_graph *g);
cpaa_status ensure_frontier(const cpaa_graph *g, Frontier &f, cpaa_graph *track);  // track: NULL or g
void free_frontier(cpaa_graph *track, Frontier &f);
cudaError_t frontier_reset(const Frontier &f, cudaStream_t st);
cudaError_t frontier_mark_nonzero(const cpaa_graph *g, const Frontier &f, int precision, int width,
                                  const void *y0, void *y1, cudaStream_t st);
cudaError_t frontier_mark_rows(const cpaa_graph *g, const Frontier &f, int count, const int32_t *rows,
                               cudaStream_t st);
cudaError_t frontier_expand(const cpaa_graph *g, const Frontier &f, int parity, cudaStream_t st);
void frontier_launch(const cpaa_graph *g, const Frontier &f, int parity, StepLaunch &sl);
cudaError_t launch_step(const StepLaunch &s);
// One round of up to 8 graphs in a single launch (same precision, width and
// stream).
cudaError_t launch_step_multi(const StepLaunch *sl, int ng);

// Solve pieces (solve.cu), shared by cpaa_solve and cpaa_solve_batch.
int stats_blocks(int64_t n);
cpaa_status ensure_reduction_buffers(cpaa_graph *g);
cpaa_status ensure_workspace(cpaa_graph *g, int prec, int width, int max_rounds);
cudaError_t launch_stats(cpaa_graph *g, const double *p, double *out, cudaStream_t st);
cpaa_status check_stats(const double *s, int64_t nnz, double *kappa);
// Prep, rounds and finalisation of one tile; with time_rounds the rounds are
// bracketed by the workspace's events, read afterwards by tile_rounds_ms
// (which waits for them).
cpaa_status run_tile(cpaa_graph *g, const TileJob &job, cudaStream_t st, bool history_all_rounds,
                     bool time_rounds);
cpaa_status tile_rounds_ms(cpaa_graph *g, float *ms);
void round_sums(int width, int b, int k, const std::vector<double> &h, double *sumT, double *sumA);

}  // namespace cpaa
