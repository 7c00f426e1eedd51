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
//   new ids [0, n_hub)  hub rows (degree > kHubDegree), by decreasing degree;
//   new ids [n_hub, n)  every other row, in windows of kSortWindow rows of the
//                       original order, each window sorted by decreasing degree.
// Every per-vertex vector (degrees, iterates, accumulator) is stored in the new
// order; the solve gathers p through the permutation and scatters pi back.
//
// Non-hub rows are held as SELL-C-sigma (sliced ELLPACK, C = kChunkRows = 32,
// sigma = kSortWindow): chunk c holds new rows n_hub + 32c .. + 31, padded to
// the chunk's longest row rounded up to a multiple of kSellVec, column-major
// in groups of kSellVec entries per lane (entry i of lane l at
// chunk_off[c] + 128 (i / 4) + 4 l + i % 4, so a warp reads 512 contiguous
// bytes per load); padding entries hold the sentinel column n, whose iterate
// value is kept at zero.  One warp owns one chunk, one lane one row.
// Windows are multiples of 32 rows, so a chunk never straddles two windows
// and its first row is its longest.
//
// Hub rows stay CSR (relabelled columns).  Their entries are cut into tiles of
// kHubTileEntries; one CTA sums one tile, and the CTA that takes the last
// ticket of a row adds the tile partials in tile order and writes the row (an
// atomic counter, no waiting).  Hub tile encoding (int4):
//   {row, tile, slot, hub + 1}   slot = partial-sum index of tile 0 of the row
// ---------------------------------------------------------------------------
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunkRows = 32;
constexpr int kSellVec = 4;     // a lane's SELL entries are stored in groups of 4 (one 16-byte load)
constexpr int kSortWindow = 1024;
constexpr int kHubDegree = 2048;
constexpr int kHubTileEntries = 2048;
constexpr int kLongChunk = 64;  // SELL chunks longer than this get a whole CTA
constexpr int kRedSlots = 256;  // atomic slots per reduced scalar and round
constexpr int kRedQ = 2;       // reduced scalars per round: sum T, sum |T|
constexpr int kDefaultMaxRounds = 2000;

constexpr int kPrepBlocks = 1024;  // CTAs of the fixed-order reductions
constexpr int kMaxWidth = 16;      // widest tile of vectors a round kernel takes

// Workspace of the solves, grown on demand and reused (one solve per graph at
// a time).  Vectors of a tile of W columns are row-major [rows x W].
struct Workspace {
    void *y0 = nullptr;        // iterates y = D^-1 T, [(n+1) x W] (row n: zero sentinel)
    void *y1 = nullptr;
    size_t vec_bytes = 0;
    void *rho = nullptr;       // accumulator D^-1 pibar, [n x W]
    void *comp = nullptr;      // Kahan compensation (FP32 paths), [n x W]
    size_t rho_bytes = 0;
    double *red = nullptr;     // per-round sums [(M+1)][2][W][kRedSlots]
    size_t red_bytes = 0;
    void *long_part = nullptr; // hub tile partials [num_hub_tiles x W]
    size_t long_part_bytes = 0;
    double *part = nullptr;    // per-CTA partials of the fixed-order reductions
    double *sums = nullptr;    // reduced scalars (device)
    double *h_sums = nullptr;  // pinned host copy of sums
    double *io = nullptr;      // device staging of host p / pi
    size_t io_bytes = 0;
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
    int num_long_chunks = 0;         // leading chunk_order entries longer than kLongChunk
    // per-vertex, new order
    double *deg64 = nullptr;         // d_u
    double *inv_deg64 = nullptr;     // 1 / d_u
    float *deg32 = nullptr;
    float *inv_deg32 = nullptr;
    int64_t device_bytes = 0;
    int tuned_width[3] = {0, 0, 0};  // batch tile width picked by the autotuner, per precision
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

// Host-side coefficient table c_0..c_M (Sec. 2.2, Proposition 1).
void cheb_coeffs(double c, int M, std::vector<double> &ck);

// Round launcher (step.cu): one round for a tile of `width` vectors.
struct StepLaunch {
    const cpaa_graph *g;
    int precision;
    int width;          // 1, 2, 4, 8 or 16
    const void *y_src;  // gathered iterates y_{k-1}, [(n+1) x width]
    void *y_io;         // in: y_{k-2} (k >= 2); out: y_k
    void *rho;          // [n x width]
    void *comp;         // [n x width]
    void *long_part;    // hub tile partials [num_hub_tiles x width]
    double *red;        // this round's [2][width][kRedSlots]
    double ck[kMaxWidth];
    unsigned active;    // columns that still accumulate
    unsigned reduce;    // columns whose sums are reduced this round
    unsigned first;     // columns in their first round (k == 1)
    int power;          // 1: power-method round (ck[b] = c, rho holds q = (1-c) p / d)
    int *long_cnt;      // hub ticket counters [n_hub], all zero; NULL = the graph's own
    cudaStream_t stream;
};
cudaError_t launch_step(const StepLaunch &s);

// Solve pieces (solve.cu), shared by cpaa_solve and cpaa_solve_batch.
int stats_blocks(int64_t n);
cpaa_status ensure_reduction_buffers(cpaa_graph *g);
cpaa_status ensure_workspace(cpaa_graph *g, int prec, int width, int max_rounds);
cudaError_t launch_stats(cpaa_graph *g, const double *p, double *out, cudaStream_t st);
cpaa_status check_stats(const double *s, int64_t nnz, double *kappa);
cpaa_status run_tile(cpaa_graph *g, const TileJob &job, cudaStream_t st, bool history_all_rounds,
                     float *rounds_ms);
void round_sums(int width, int b, int k, const std::vector<double> &h, double *sumT, double *sumA);

}  // namespace cpaa
