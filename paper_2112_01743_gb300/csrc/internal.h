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
// Tiling of the step kernels.
//
// The rows are cut into tiles of at most kTileItems "merge-path items", an
// item being either one CSR entry or one row end.  A block tile holds whole
// consecutive rows; one CTA owns it and writes every row of it.  A row whose
// degree + 1 exceeds kTileItems is a long row: its entries are cut into
// chunks of kTileItems; each chunk is one tile, and the CTA that finishes the
// last chunk of a row (an atomic ticket, no waiting) adds the chunk partials
// in chunk order and writes the row.
//
// Tile encoding (int4):
//   block tile: {r0, r1, 0, 0}                  rows [r0, r1)
//   chunk tile: {row, chunk, slot, long_id + 1} slot = partial-sum index of
//                                               chunk 0 of this row
// Chunk tiles come first so the heaviest rows start first.
// ---------------------------------------------------------------------------
constexpr int kThreads = 256;
constexpr int kItemsPerThread = 8;
constexpr int kTileItems = kThreads * kItemsPerThread;  // 2048
constexpr int kMaxTileRows = kTileItems / 2;            // every row holds >= 1 entry
constexpr int kRedSlots = 64;  // atomic slots per reduced scalar and round
constexpr int kRedQ = 3;       // reduced scalars per round: sum T, sum |T|, sum d*pibar
constexpr int kDefaultMaxRounds = 2000;

// Workspace for one single-vector solve, sized for one precision at a time.
struct Workspace {
    int precision = -1;
    size_t vec_bytes = 0;   // bytes of one iterate vector
    void *y0 = nullptr;     // iterate buffers (y = D^-1 T, see step.cu)
    void *y1 = nullptr;
    void *rho = nullptr;    // accumulator D^-1 pibar (FP64 or FP32)
    void *comp = nullptr;   // Kahan compensation (FP32 paths)
    double *red = nullptr;  // [(max_rounds+1)][kRedQ][kRedSlots]
    int red_rounds = 0;
    double *prep_part = nullptr;  // per-CTA partials of the prep reduction
    double *prep_out = nullptr;   // 4 reduced scalars
    double *h_prep = nullptr;     // pinned host copy of prep_out
    double *d_pi = nullptr;       // device output when pi is a host pointer
    double *d_p = nullptr;        // device input when p is a host pointer
};

}  // namespace cpaa

struct cpaa_graph {
    int64_t n = 0;
    int64_t nnz = 0;
    int device = 0;
    int32_t *row_ptr = nullptr;   // device [n+1]
    int32_t *col_idx = nullptr;   // device [nnz + 4], zero padded for 16-byte loads
    double *deg64 = nullptr;      // d_u
    double *inv_deg64 = nullptr;  // 1 / d_u
    float *deg32 = nullptr;
    float *inv_deg32 = nullptr;
    int4 *tiles = nullptr;
    int num_tiles = 0;
    int num_chunk_tiles = 0;
    int num_long = 0;
    int total_chunks = 0;
    double *long_part = nullptr;  // chunk partial sums [total_chunks] (FP64 or FP32 view)
    int *long_cnt = nullptr;      // per long row ticket counter [num_long], kept at zero
    int64_t device_bytes = 0;
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

// Step launchers (step.cu).
struct StepLaunch {
    const cpaa_graph *g;
    int precision;
    const void *y_src;  // gathered iterate y_{k-1}
    void *y_io;         // in: y_{k-2} (k >= 2); out: y_k
    void *rho;
    void *comp;
    double *red;        // this round's [kRedQ][kRedSlots]
    double ck;
    int first;          // k == 1
    int last;           // also reduce sum d*pibar
    cudaStream_t stream;
};
cudaError_t launch_step(const StepLaunch &s);

}  // namespace cpaa
