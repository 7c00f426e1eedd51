// server.cu -- cpaa_server_*: continuous batching of personalised PageRank
// queries over resident graphs (see cpaa.h).
//
// Per graph: W column slots, one CUDA stream, a FIFO of queued queries.  The
// slots' vectors form one row-major [(n+1) x w] tile (the same layout and
// round kernel as cpaa_solve_batch) whose width w is the smallest power of
// two covering the highest live slot: queries take the lowest free slot, so
// at low load a lone query runs at w = 1 (a compact, cache-resident iterate)
// and under load the tile widens to W.  When w changes between rounds, a copy
// kernel moves the live columns, bit for bit, into a spare buffer at the new
// stride.  Two host threads:
//   scheduler   - admits queued queries into free slots between rounds (a new
//                 column's y_0 goes into the buffer the next round gathers
//                 from, y[G & 1] after G rounds, so every column follows the
//                 tile's ping-pong parity), launches one round per graph with
//                 per-column first/active masks and coefficients, and after a
//                 column's last round queues its finalisation;
//   completion  - waits for a finished column's finalisation and marks the
//                 query done; its vector stays in the slot's device buffer
//                 until cpaa_server_wait copies it out and frees the slot (an
//                 uncollected result holds its slot: back-pressure).
// At most kInFlight rounds per graph are queued ahead of the device, so new
// queries join quickly.  Each column's arithmetic is the same whatever the
// other columns hold, so a result is bit-identical alone and in a mix.
//
// Fused mode (CPAA_SERVER_FUSED): all graphs share one stream, and each
// scheduling pass launches the rounds of every graph with live columns as one
// kernel over the graphs' work lists (launch_step_multi); the per-graph host
// logic is the same.
//
// With the a-posteriori stopping rule every round also takes its per-column
// sums and tests the rule on the device (step.cu); a column that passes stops
// accumulating at once.  After each round a one-warp kernel writes the stop
// state to mapped host memory, and the scheduler, which reads it when the
// round's event completes (a lag of at most kInFlight rounds), finalises the
// column.
// The rule's decision uses only that column's sums, so it too is the same
// alone and in a mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <limits>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "device_common.cuh"

namespace cpaa {
namespace srv {

using clk = std::chrono::steady_clock;
constexpr int kInFlight = 4;
constexpr int kMaxFusedGraphs = 8;  // graphs per fused round launch
constexpr size_t kMaxQueue = size_t(1) << 20;

__device__ __forceinline__ void sput(double *p, double v) { *p = v; }
__device__ __forceinline__ void sput(float *p, double v) { *p = __double2float_rn(v); }
__device__ __forceinline__ void sput(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }
__device__ __forceinline__ double sget(const double *p) { return *p; }
__device__ __forceinline__ double sget(const float *p) { return (double)*p; }
__device__ __forceinline__ double sget(const __nv_bfloat16 *p) { return (double)__bfloat162float(*p); }
__device__ __forceinline__ void sput(df *p, double v) { *p = df(v); }
__device__ __forceinline__ double sget(const df *p) { return __dadd_rn((double)p->hi, (double)p->lo); }

// Stop state of a graph's columns under the a-posteriori rule (device, and
// pinned host copies of it).
struct DevStop {
    unsigned stop;                // stopped columns
    int round[kMaxWidth];         // the round a column stopped after (-1: running)
    double maxl1[kMaxWidth];      // running max of ||T_j p||_1
};

struct SeedArgs {
    int count;
    int col;
    double c0half;
    double l1;                    // ||p||_1, the rule's starting max
    int32_t r[CPAA_SERVER_MAX_SEEDS];  // new ids
    double w[CPAA_SERVER_MAX_SEEDS];
};

// Column b of a new query: y_0 = D^-1 p, rho = (c_0/2) y_0, comp = 0, with p
// zero outside the seeds (same arithmetic as the dense prep of solve.cu).
template <class S, class R, int W>
__global__ void slot_zero_kernel(S *y0, S *y1, R *rho, R *comp, int64_t n, int b) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        y0[u * W + b] = S(0.0f);
        if (y1) y1[u * W + b] = S(0.0f);  // sparse-frontier start: rows outside the ball stay +0
        rho[u * W + b] = R(0);
        if (comp) comp[u * W + b] = R(0);
    }
}

// A tile's array at a new width: dst[r][b] = src[r][b] for the kept columns b
// of both widths, 0 elsewhere (the sentinel row stays zero).  Raw element bits
// are copied, so a moved column continues exactly as it would have.
template <class E>
__global__ void restride_kernel(const E *__restrict__ src, E *__restrict__ dst, int64_t rows, int wo_log,
                                int wn_log, unsigned keep) {
    const int64_t total = rows << wn_log;
    const int64_t bmask = (int64_t(1) << wn_log) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i & bmask);
        E v = E(0);
        if ((keep >> b & 1u) && b < (1 << wo_log)) v = src[((i >> wn_log) << wo_log) + b];
        dst[i] = v;
    }
}

// Copy the stop state into mapped host memory (read by the host once an
// event after this kernel has completed).
__global__ void copy_stop_kernel(const DevStop *__restrict__ src, DevStop *dst) {
    const unsigned *s = reinterpret_cast<const unsigned *>(src);
    unsigned *d = reinterpret_cast<unsigned *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(DevStop) / 4); i += blockDim.x) d[i] = s[i];
}

template <class S, class R, int W>
__global__ void slot_seed_kernel(const SeedArgs a, const double *__restrict__ inv64, S *y0, R *rho,
                                 DevStop *ds) {
    const int i = threadIdx.x;
    if (i == 0 && ds) {  // the column starts running under the a-posteriori rule
        ds->stop &= ~(1u << a.col);
        ds->round[a.col] = -1;
        ds->maxl1[a.col] = a.l1;
    }
    if (i < a.count) {
        const int64_t u = a.r[i];
        sput(y0 + u * W + a.col, __dmul_rn(a.w[i], inv64[u]));
        sput(rho + u * W + a.col, __dmul_rn(a.c0half, sget(y0 + u * W + a.col)));
    }
}

// Normaliser of column b (fixed order, as in solve.cu) and the finalisation
// into out (caller's order).
template <class R, int W>
__global__ void __launch_bounds__(kThreads) col_norm_kernel(const R *__restrict__ rho,
                                                            const double *__restrict__ deg64,
                                                            int64_t n, int b, double *part) {
    __shared__ double s[kThreads];
    double v = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)kThreads + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreads)
        v = __fma_rn(deg64[u], sget(rho + u * W + b), v);
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = __dadd_rn(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(kThreads) col_sum_kernel(const double *part, int nblocks, double *out) {
    __shared__ double s[kThreads];
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) v = __dadd_rn(v, part[b]);
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = __dadd_rn(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

template <class R, int W>
__global__ void __launch_bounds__(kThreads) col_finalize_kernel(const R *__restrict__ rho,
                                                                const double *__restrict__ deg64,
                                                                const int32_t *__restrict__ perm,
                                                                int64_t n, int b, const double *sum,
                                                                int normalize, double one_minus_c,
                                                                double *out) {
    const double scale = normalize == 0 ? __drcp_rn(*sum) : one_minus_c;
    for (int64_t u = blockIdx.x * (int64_t)kThreads + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * kThreads)
        out[perm[u]] = __dmul_rn(scale, __dmul_rn(deg64[u], sget(rho + u * W + b)));
}

struct GraphState;
struct Request {
    uint64_t ticket = 0;
    int graph = 0;
    SeedArgs seeds{};
    double c = 0, tol = 0, kappa = 0;
    int M = 0;
    bool notconv = false;
    bool by_posteriori = false;  // stopped by the a-posteriori rule at round M
    double maxl1 = 0;            // that rule's running max at the stop
    enum State { PENDING, RUNNING, DONE, CANCELLED } state = PENDING;
    bool cancel = false;
    bool collecting = false;  // cpaa_server_wait is copying the result out
    bool spilling = false;    // the completion thread is moving it to host memory
    GraphState *gs = nullptr; // where the result waits (state DONE), or NULL once spilled
    int slot = -1;
    std::vector<double> host; // the result after a spill
    clk::time_point t_submit, t_admit, t_done;
};
using ReqP = std::shared_ptr<Request>;

enum SlotState { FREE, LIVE, FINISHING, READY };
struct Slot {
    ReqP req;
    int k = 0;
    SlotState st = FREE;
    std::vector<double> ck;
    cudaEvent_t done = nullptr;
    int64_t g_admit = 0;         // the graph's round count when the query was admitted
};

struct GraphState {
    int id = 0;
    cpaa_graph *g = nullptr;
    int W = 1;  // slots
    int w = 1;  // current tile width (a power of two, 1..W)
    cudaStream_t stream = nullptr;
    // y, rho, comp and spare: interchangeable buffers of tile_bytes(g, prec, W) each
    void *y[2] = {nullptr, nullptr};
    void *rho = nullptr, *comp = nullptr, *spare = nullptr, *long_part = nullptr;
    int *long_cnt = nullptr;
    double *red = nullptr, *result = nullptr, *part = nullptr, *sums = nullptr;
    size_t bytes = 0;
    std::vector<int32_t> inv_perm;  // caller id -> new id
    std::vector<double> deg;        // caller order
    std::vector<Slot> slots;
    std::deque<ReqP> pending;
    bool own_stream = true;
    int64_t G = 0;       // rounds launched
    int64_t G_seen = 0;  // rounds whose completion the scheduler has processed
    cudaEvent_t ring[kInFlight] = {};
    // a-posteriori rule (NULL otherwise)
    double *ipart = nullptr, *ipart2 = nullptr;
    DevStop *dstop = nullptr;
    // mapped host memory, written by copy_stop_kernel (no copy engine: a
    // per-round copy would queue behind large result copies)
    DevStop *h_ring = nullptr;  // [kInFlight]: stop state after round r at r % kInFlight
    DevStop *h_slot = nullptr;  // [W]: stop state at each slot's finalisation
    DevStop *d_ring = nullptr;  // device addresses of the same memory
    DevStop *d_slot = nullptr;
    // sparse frontier (CPAA_SPARSE_FRONTIER): a tile that starts from empty runs
    // its early rounds on the ball of its queries' seeds, until a query joins
    // the running ones, the ball is large, or kFrontierRounds have run
    Frontier fr;
    bool fr_ok = false;  // the frontier is allocated for this graph (it is large enough to gain)
    bool fr_on = false;  // the current rounds run on the frontier
    int fr_k = 0;        // frontier rounds run since it started
};

struct Completion {
    GraphState *gs;
    int slot;
    ReqP req;
    bool spill;  // move a finished, uncollected result to host memory
};

}  // namespace srv
}  // namespace cpaa

using namespace cpaa;
using namespace cpaa::srv;

struct cpaa_server {
    size_t budget = 0, used = 0;
    int prec = CPAA_F32, normalize = 0, max_rounds = kDefaultMaxRounds;
    int posteriori = 0;  // stop rule CPAA_STOP_POSTERIORI
    int fused = 0;       // CPAA_SERVER_FUSED: one stream, one round launch over all graphs
    int frontier = 0;    // CPAA_SPARSE_FRONTIER (not with CPAA_SERVER_FUSED)
    cudaStream_t fstream = nullptr;
    int device = 0;
    std::vector<std::unique_ptr<GraphState>> graphs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_comp;
    std::unordered_map<uint64_t, ReqP> reqs;
    uint64_t next_ticket = 1;
    std::deque<Completion> comps;
    std::thread sched, comp_th;
    bool stop = false;
    cudaStream_t copy_stream = nullptr;
    std::mutex copy_mu;
    uint64_t submitted = 0, completed = 0, cancelled = 0, failed = 0;
    std::atomic<uint64_t> rounds{0}, round_columns{0}, relayouts{0};
    std::vector<double> lat_us, admit_us;
};

namespace cpaa {
namespace srv {

static size_t vbytes(int prec) { return prec == CPAA_F64 || prec == CPAA_DF64 ? 8 : prec == CPAA_F32 ? 4 : 2; }
static size_t rbytes(int prec) { return prec == CPAA_F64 || prec == CPAA_DF64 ? 8 : 4; }

// Bytes of each of a tile's five vector buffers (y[0], y[1], rho, comp, spare).
static size_t tile_bytes(const cpaa_graph *g, int prec, int W) {
    const size_t n = (size_t)g->n;
    return std::max((n + 1) * W * vbytes(prec), n * W * rbytes(prec));
}

// Graphs below this many entries serve without the sparse frontier: their
// rounds are chains of launch latencies, which two more kernels per round lengthen.
constexpr int64_t kFrontierMinEntries = int64_t(1) << 22;

static size_t graph_bytes(const cpaa_graph *g, int prec, int W, int posteriori, int frontier) {
    const size_t n = (size_t)g->n;
    size_t b = 5 * tile_bytes(g, prec, W) + n * W * 8 +
               (size_t)std::max(1, g->num_hub_tiles) * W * 8 + (size_t)std::max(1, g->n_hub) * 4 +
               (size_t)kPrepBlocks * 8 + (size_t)W * 8 + 2 * 8 * (size_t)W;
    if (posteriori)  // per-round item sums
        b += 2 * 8 * (size_t)W * ((size_t)g->n_hub + g->num_chunks + kSumBlocks) + sizeof(DevStop);
    if (frontier && g->nnz >= kFrontierMinEntries) b += frontier_bytes(g);
    return b;
}

template <class S, class R, int W>
static void launch_slot_prep(GraphState &gs, int b, const SeedArgs &a, bool both) {
    const int64_t n = gs.g->n;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 2048);
    R *comp = std::is_same<R, float>::value ? (R *)gs.comp : nullptr;
    S *y0 = (S *)gs.y[gs.G & 1];  // the buffer the next round gathers from
    S *y1 = both ? (S *)gs.y[(gs.G + 1) & 1] : nullptr;
    slot_zero_kernel<S, R, W><<<grid, 256, 0, gs.stream>>>(y0, y1, (R *)gs.rho, comp, n, b);
    slot_seed_kernel<S, R, W><<<1, CPAA_SERVER_MAX_SEEDS, 0, gs.stream>>>(a, gs.g->inv_deg64, y0, (R *)gs.rho,
                                                                         gs.dstop);
}

template <class R, int W>
static void launch_slot_final(GraphState &gs, int b, int normalize, double c) {
    const int64_t n = gs.g->n;
    const int blocks = stats_blocks(n);
    const unsigned grid = (unsigned)std::min<int64_t>((n + kThreads - 1) / kThreads, 8192);
    col_norm_kernel<R, W><<<blocks, kThreads, 0, gs.stream>>>((const R *)gs.rho, gs.g->deg64, n, b, gs.part);
    col_sum_kernel<<<1, kThreads, 0, gs.stream>>>(gs.part, blocks, gs.sums + b);
    col_finalize_kernel<R, W><<<grid, kThreads, 0, gs.stream>>>((const R *)gs.rho, gs.g->deg64, gs.g->perm, n, b,
                                                               gs.sums + b, normalize, 1.0 - c,
                                                               gs.result + (size_t)b * n);
}

template <class S, class R>
static void slot_prep_w(GraphState &gs, int b, const SeedArgs &a, bool both) {
    switch (gs.w) {
        case 1: launch_slot_prep<S, R, 1>(gs, b, a, both); break;
        case 2: launch_slot_prep<S, R, 2>(gs, b, a, both); break;
        case 4: launch_slot_prep<S, R, 4>(gs, b, a, both); break;
        case 8: launch_slot_prep<S, R, 8>(gs, b, a, both); break;
        case 16: launch_slot_prep<S, R, 16>(gs, b, a, both); break;
    }
}

template <class R>
static void slot_final_w(GraphState &gs, int b, int normalize, double c) {
    switch (gs.w) {
        case 1: launch_slot_final<R, 1>(gs, b, normalize, c); break;
        case 2: launch_slot_final<R, 2>(gs, b, normalize, c); break;
        case 4: launch_slot_final<R, 4>(gs, b, normalize, c); break;
        case 8: launch_slot_final<R, 8>(gs, b, normalize, c); break;
        case 16: launch_slot_final<R, 16>(gs, b, normalize, c); break;
    }
}

static void slot_prep(cpaa_server *s, GraphState &gs, int b, const SeedArgs &a, bool both) {
    if (s->prec == CPAA_F64) slot_prep_w<double, double>(gs, b, a, both);
    else if (s->prec == CPAA_F32) slot_prep_w<float, float>(gs, b, a, both);
    else if (s->prec == CPAA_DF64) slot_prep_w<df, df>(gs, b, a, both);
    else slot_prep_w<__nv_bfloat16, float>(gs, b, a, both);
}

static void slot_final(cpaa_server *s, GraphState &gs, int b, double c) {
    if (s->prec == CPAA_F64) slot_final_w<double>(gs, b, s->normalize, c);
    else if (s->prec == CPAA_DF64) slot_final_w<df>(gs, b, s->normalize, c);
    else slot_final_w<float>(gs, b, s->normalize, c);
    // the column's stop state as of its finalisation (read by the completion thread)
    if (gs.dstop) copy_stop_kernel<<<1, 64, 0, gs.stream>>>(gs.dstop, gs.d_slot + b);
}

static int log2_width(int w) {
    int l = 0;
    while ((1 << l) < w) ++l;
    return l;
}

template <class E>
static void restride(GraphState &gs, void *&buf, int64_t rows, int wn, unsigned keep) {
    const int64_t total = rows * wn;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096));
    restride_kernel<E><<<grid, 256, 0, gs.stream>>>((const E *)buf, (E *)gs.spare, rows, log2_width(gs.w),
                                                     log2_width(wn), keep);
    std::swap(buf, gs.spare);
}

// EY: the iterate's element (bits), ER: the accumulator's; comp is kept only
// under Kahan summation (FP32 accumulators).
template <class EY, class ER>
static void restride_arrays(GraphState &gs, int wn, unsigned keep, bool kahan) {
    const int64_t n = gs.g->n;
    restride<EY>(gs, gs.y[0], n + 1, wn, keep);
    restride<EY>(gs, gs.y[1], n + 1, wn, keep);
    restride<ER>(gs, gs.rho, n, wn, keep);
    if (kahan) restride<ER>(gs, gs.comp, n, wn, keep);
}

// Change a graph's tile width to wn between rounds (stream-ordered after every
// kernel already queued on the graph's stream), keeping the columns in keep.
static void set_width(cpaa_server *s, GraphState &gs, int wn, unsigned keep) {
    if (wn == gs.w) return;
    using u64 = unsigned long long;
    switch (s->prec) {
        case CPAA_F64:
        case CPAA_DF64: restride_arrays<u64, u64>(gs, wn, keep, false); break;
        case CPAA_F32: restride_arrays<uint32_t, uint32_t>(gs, wn, keep, true); break;
        default: restride_arrays<uint16_t, uint32_t>(gs, wn, keep, true); break;  // BF16
    }
    gs.w = wn;
    ++s->relayouts;
}

// Queue a LIVE slot's finalisation and hand it to the completion thread
// (caller does not hold s->mu).
static void finish_slots(cpaa_server *s, GraphState &gs, const std::vector<int> &cols) {
    if (cols.empty()) return;
    std::vector<Completion> done;
    for (int b : cols) {
        Slot &slot = gs.slots[b];
        slot_final(s, gs, b, slot.req->c);
        cudaEventRecord(slot.done, gs.stream);
        done.push_back({&gs, b, slot.req, false});
    }
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &c : done) {
        gs.slots[c.slot].st = FINISHING;
        s->comps.push_back(c);
    }
    s->cv_comp.notify_one();
}

// Rounds that completed since the last pass: under the a-posteriori rule, the
// columns they stopped are finalised now.  A view counts for a slot only if it
// was taken after the slot's query was admitted (its prep reset the column).
static void process_completed_rounds(cpaa_server *s, GraphState &gs) {
    std::vector<int> stopped;
    while (gs.G_seen < gs.G) {
        const int64_t r = gs.G_seen + 1;
        if (cudaEventQuery(gs.ring[r % kInFlight]) != cudaSuccess) break;
        if (gs.h_ring) {
            const DevStop &v = gs.h_ring[r % kInFlight];
            // slot states are also changed by the completion thread and waiters
            std::lock_guard<std::mutex> lk(s->mu);
            for (int b = 0; b < gs.W; ++b) {
                const Slot &sl = gs.slots[b];
                if (sl.st == LIVE && (v.stop >> b & 1u) && r > sl.g_admit &&
                    std::find(stopped.begin(), stopped.end(), b) == stopped.end())
                    stopped.push_back(b);
            }
        }
        gs.G_seen = r;
    }
    finish_slots(s, gs, stopped);
}

static double us_since(clk::time_point a, clk::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
}

// The host side of a graph's next round: completed rounds processed,
// cancellations and admissions made, and (if any column is live) the round's
// launch described in sl.  Returns true when sl is to be launched; *admitted_any
// tells whether queries joined.
static bool plan_round(cpaa_server *s, GraphState &gs, StepLaunch &sl, unsigned *live_out, bool *admitted_any) {
    *admitted_any = false;
    process_completed_rounds(s, gs);
    // at most kInFlight rounds queued: launch G+1 waits until round G+1-kInFlight
    // has completed and been processed (its ring entry is then free)
    if (gs.G + 1 > kInFlight && gs.G_seen < gs.G + 1 - kInFlight) return false;
    std::vector<std::pair<int, SeedArgs>> admitted;
    unsigned live = 0, live_before = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const auto now = clk::now();
        for (int b = 0; b < gs.W; ++b) {
            Slot &sl = gs.slots[b];
            if (sl.st == LIVE && sl.req->cancel) {
                sl.req->state = Request::CANCELLED;
                sl.req->t_done = now;
                ++s->cancelled;
                sl.req.reset();
                sl.st = FREE;
                s->cv_done.notify_all();
            }
        }
        for (int b = 0; b < gs.W; ++b)
            if (gs.slots[b].st == LIVE) live_before |= 1u << b;
        {
            for (int b = 0; b < gs.W && !gs.pending.empty(); ++b) {
                Slot &sl = gs.slots[b];
                if (sl.st != FREE) continue;
                ReqP r;
                while (!gs.pending.empty() && !r) {
                    r = gs.pending.front();
                    gs.pending.pop_front();
                    if (r->cancel) {  // cancelled while queued
                        r->state = Request::CANCELLED;
                        r->t_done = now;
                        ++s->cancelled;
                        s->cv_done.notify_all();
                        r.reset();
                    }
                }
                if (!r) break;
                sl.req = r;
                sl.k = 0;
                sl.st = LIVE;
                sl.g_admit = gs.G;
                cheb_coeffs(r->c, r->M, sl.ck);
                r->state = Request::RUNNING;
                r->t_admit = now;
                s->admit_us.push_back(us_since(r->t_submit, now));
                SeedArgs a = r->seeds;
                a.col = b;
                a.c0half = sl.ck[0] / 2.0;
                admitted.emplace_back(b, a);
            }
        }
        for (int b = 0; b < gs.W; ++b)
            if (gs.slots[b].st == LIVE) live |= 1u << b;
        // queued queries but no free slot: spill uncollected results to host memory
        if (!gs.pending.empty()) {
            bool any_free = false;
            for (auto &sl : gs.slots) any_free |= sl.st == FREE;
            if (!any_free) {
                bool queued = false;
                for (int b = 0; b < gs.W; ++b) {
                    Slot &sl = gs.slots[b];
                    if (sl.st == READY && !sl.req->collecting && !sl.req->spilling) {
                        sl.req->spilling = true;
                        s->comps.push_back({&gs, b, sl.req, true});
                        queued = true;
                    }
                }
                if (queued) s->cv_comp.notify_one();
            }
        }
    }
    if (live) {  // the narrowest tile that holds every live column
        const int need = 32 - __builtin_clz(live);
        int wn = 1;
        while (wn < need) wn <<= 1;
        set_width(s, gs, wn, live);
    }
    // sparse frontier: a tile that starts from empty starts on the ball of its
    // queries' seeds; a query that joins running ones ends the frontier rounds
    // (its seeds are outside the ball the others have grown)
    const bool fr_start = gs.fr_ok && live_before == 0 && !admitted.empty();
    if (!admitted.empty() && !fr_start) gs.fr_on = false;
    if (fr_start) {
        frontier_reset(gs.fr, gs.stream);
        if (gs.ipart)  // items the early rounds skip keep a zero partial-sum slot
            cudaMemsetAsync(gs.ipart, 0, 2 * 8 * (size_t)gs.W * ((size_t)gs.g->n_hub + gs.g->num_chunks),
                            gs.stream);
        gs.fr_on = true;
        gs.fr_k = 0;
    }
    for (auto &a : admitted) {
        slot_prep(s, gs, a.first, a.second, fr_start);
        if (fr_start) frontier_mark_rows(gs.g, gs.fr, a.second.count, a.second.r, gs.stream);
    }
    *admitted_any = !admitted.empty();
    *live_out = live;
    if (!live) return false;

    sl = StepLaunch();
    sl.g = gs.g;
    sl.precision = s->prec;
    sl.width = gs.w;
    sl.y_src = gs.y[gs.G & 1];
    sl.y_io = gs.y[(gs.G + 1) & 1];
    sl.rho = gs.rho;
    sl.comp = gs.comp;
    sl.long_part = gs.long_part;
    sl.red = gs.red;
    sl.active = live;
    sl.reduce = 0;
    sl.first = ~live & ((1u << gs.w) - 1u);
    sl.power = 0;
    // no deferred accumulation (StepLaunch::pend): a tile's width, and with it
    // the kernel form, may change between two rounds of a query
    sl.long_cnt = gs.long_cnt;
    sl.stream = gs.stream;
    for (int b = 0; b < kMaxWidth; ++b) sl.ck[b] = 0.0;
    for (int b = 0; b < gs.W; ++b) {
        if (!(live >> b & 1u)) continue;
        const int k = gs.slots[b].k + 1;  // this column's round
        sl.ck[b] = gs.slots[b].ck[k];
        if (k == 1) sl.first |= 1u << b;
    }
    if (gs.dstop) {
        // every round takes its sums and tests the a-posteriori rule
        sl.ipart = gs.ipart;
        sl.ipart2 = gs.ipart2;
        sl.reduce = live;
        sl.stop = &gs.dstop->stop;
        sl.sa.decide = live;
        for (int b = 0; b < gs.W; ++b) {
            if (!(live >> b & 1u)) continue;
            const Slot &slot = gs.slots[b];
            sl.sa.k[b] = slot.k + 1;
            sl.sa.err[b] = err_bound(slot.req->c, slot.k + 1);
            sl.sa.tol[b] = slot.req->tol;
        }
        sl.sa.normalize = s->normalize;
        sl.sa.maxl1 = gs.dstop->maxl1;
        sl.sa.stop = &gs.dstop->stop;
        sl.sa.stop_round = gs.dstop->round;
    }
    if (gs.fr_on) {
        if (gs.fr_k < kFrontierRounds) {
            ++gs.fr_k;
            frontier_expand(gs.g, gs.fr, gs.fr_k, gs.stream);
            frontier_launch(gs.g, gs.fr, gs.fr_k, sl);
        } else {
            gs.fr_on = false;
        }
    }
    return true;
}

// The host side after a graph's round was launched: the stop state copied
// out, the round counted, and columns at their last round finalised.
static void after_round(cpaa_server *s, GraphState &gs, unsigned live) {
    const int64_t Gn = gs.G + 1;
    if (gs.dstop)
        copy_stop_kernel<<<1, 64, 0, gs.stream>>>(gs.dstop, gs.d_ring + Gn % kInFlight);
    gs.G = Gn;
    ++s->rounds;
    s->round_columns += (uint64_t)gs.w;
    cudaEventRecord(gs.ring[gs.G % kInFlight], gs.stream);
    std::vector<int> due;
    for (int b = 0; b < gs.W; ++b) {
        if (!(live >> b & 1u)) continue;
        if (++gs.slots[b].k == gs.slots[b].req->M) due.push_back(b);
    }
    finish_slots(s, gs, due);
}

// One scheduling pass over a graph with its own stream; true if anything was
// launched.
static bool step_graph(cpaa_server *s, GraphState &gs) {
    StepLaunch sl;
    unsigned live = 0;
    bool admitted = false;
    if (!plan_round(s, gs, sl, &live, &admitted)) return admitted;
    if (launch_step(sl) != cudaSuccess) return admitted;
    after_round(s, gs, live);
    return true;
}

// Fused mode: one scheduling pass over every graph, their rounds launched
// together (one kernel per group of up to kMaxFusedGraphs graphs of one tile
// width) on the server's single stream.
static bool step_fused(cpaa_server *s, const std::vector<GraphState *> &gl) {
    std::vector<StepLaunch> sls;
    std::vector<std::pair<GraphState *, unsigned>> parts;
    bool any = false;
    for (auto *gs : gl) {
        StepLaunch sl;
        unsigned live = 0;
        bool admitted = false;
        if (plan_round(s, *gs, sl, &live, &admitted)) {
            sls.push_back(sl);
            parts.push_back({gs, live});
        }
        any |= admitted;
    }
    if (sls.empty()) return any;
    std::vector<char> done(sls.size(), 0);
    for (size_t i = 0; i < sls.size(); ++i) {
        if (done[i]) continue;
        std::vector<StepLaunch> group;
        std::vector<size_t> members;
        for (size_t j = i; j < sls.size() && (int)group.size() < kMaxFusedGraphs; ++j)
            if (!done[j] && sls[j].width == sls[i].width) {
                group.push_back(sls[j]);
                members.push_back(j);
                done[j] = 1;
            }
        if (launch_step_multi(group.data(), (int)group.size()) != cudaSuccess) continue;
        for (size_t j : members) after_round(s, *parts[j].first, parts[j].second);
    }
    return true;
}

static void scheduler_main(cpaa_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<GraphState *> gl;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto busy = [&]() {
                for (auto &g : s->graphs) {
                    if (!g->pending.empty()) return true;
                    for (auto &sl : g->slots)
                        if (sl.st == LIVE) return true;
                }
                return false;
            };
            s->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&]() { return s->stop || busy(); });
            if (s->stop) return;
            for (auto &g : s->graphs) gl.push_back(g.get());
        }
        bool progressed = false;
        if (s->fused) {
            progressed = step_fused(s, gl);
        } else {
            for (auto *g : gl) progressed |= step_graph(s, *g);
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

static void completion_main(cpaa_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        Completion c;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_comp.wait(lk, [&]() { return s->stop || !s->comps.empty(); });
            if (s->comps.empty()) return;  // stop requested and nothing left
            c = s->comps.front();
            s->comps.pop_front();
        }
        GraphState &gs = *c.gs;
        if (c.spill) {
            const int64_t n = gs.g->n;
            std::vector<double> h((size_t)n);
            cudaError_t e;
            {
                std::lock_guard<std::mutex> ck(s->copy_mu);
                e = cudaMemcpyAsync(h.data(), gs.result + (size_t)c.slot * n, sizeof(double) * n,
                                    cudaMemcpyDeviceToHost, s->copy_stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
            }
            std::lock_guard<std::mutex> lk(s->mu);
            c.req->spilling = false;
            if (e == cudaSuccess && c.req->state == Request::DONE && c.req->gs == &gs) {
                c.req->host.swap(h);
                Slot &sl = gs.slots[c.slot];
                sl.req.reset();
                sl.st = FREE;
                c.req->gs = nullptr;
                c.req->slot = -1;
                s->cv_work.notify_one();
            }
            s->cv_done.notify_all();
            continue;
        }
        const cudaError_t e = cudaEventSynchronize(gs.slots[c.slot].done);
        std::lock_guard<std::mutex> lk(s->mu);
        const auto now = clk::now();
        c.req->t_done = now;
        if (e == cudaSuccess && gs.h_slot) {
            const DevStop &v = gs.h_slot[c.slot];
            if ((v.stop >> c.slot & 1u) && v.round[c.slot] >= 1 && v.round[c.slot] <= c.req->M) {
                c.req->M = v.round[c.slot];
                c.req->by_posteriori = true;
                c.req->maxl1 = v.maxl1[c.slot];
                c.req->notconv = false;
            }
        }
        if (e == cudaSuccess) {
            c.req->state = Request::DONE;
            c.req->gs = &gs;
            c.req->slot = c.slot;
            gs.slots[c.slot].st = READY;
            ++s->completed;
            s->lat_us.push_back(us_since(c.req->t_submit, now));
        } else {
            c.req->state = Request::CANCELLED;
            gs.slots[c.slot].req.reset();
            gs.slots[c.slot].st = FREE;
            ++s->failed;
            s->cv_work.notify_one();
        }
        s->cv_done.notify_all();
    }
}

// Free a READY slot (caller holds s->mu).
static void release_slot(cpaa_server *s, Request &r) {
    if (r.gs && r.slot >= 0) {
        Slot &sl = r.gs->slots[r.slot];
        sl.req.reset();
        sl.st = FREE;
        r.gs = nullptr;
        r.slot = -1;
        s->cv_work.notify_one();
    }
}

static void free_graph_state(GraphState &gs) {
    cudaFree(gs.y[0]); cudaFree(gs.y[1]); cudaFree(gs.rho); cudaFree(gs.comp); cudaFree(gs.spare);
    cudaFree(gs.long_part);
    cudaFree(gs.long_cnt); cudaFree(gs.red); cudaFree(gs.result); cudaFree(gs.part); cudaFree(gs.sums);
    cudaFree(gs.ipart); cudaFree(gs.ipart2); cudaFree(gs.dstop);
    free_frontier(nullptr, gs.fr);
    if (gs.h_ring) cudaFreeHost(gs.h_ring);
    if (gs.h_slot) cudaFreeHost(gs.h_slot);
    for (auto &e : gs.ring) if (e) cudaEventDestroy(e);
    for (auto &sl : gs.slots) if (sl.done) cudaEventDestroy(sl.done);
    if (gs.stream && gs.own_stream) cudaStreamDestroy(gs.stream);
}

static double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
}

}  // namespace srv
}  // namespace cpaa

extern "C" cpaa_status cpaa_server_create(size_t device_mem_budget, const cpaa_options *opt,
                                          cpaa_server **out) {
    clear_error();
    if (!out) return fail(CPAA_EINVAL, "out is NULL");
    *out = nullptr;
    cpaa_options o;
    if (opt) o = *opt;
    else {
        cpaa_options_init(&o);
        o.precision = CPAA_F32;
    }
    if (o.precision != CPAA_F64 && o.precision != CPAA_F32 && o.precision != CPAA_BF16 &&
        o.precision != CPAA_DF64)
        return fail(CPAA_EINVAL, "unknown precision");
    if (o.normalize != 0 && o.normalize != 1) return fail(CPAA_EINVAL, "normalize must be 0 or 1");
    if (o.stop_rule != CPAA_STOP_RIGOROUS && o.stop_rule != CPAA_STOP_POSTERIORI)
        return fail(CPAA_EINVAL, "unknown stop_rule");
    if (o.flags & (CPAA_INTERVAL | CPAA_CERTIFY_INTERVAL))
        return fail(CPAA_EINVAL, "the server runs the series on [-1, 1] only (no CPAA_INTERVAL / CPAA_CERTIFY_INTERVAL)");
    cpaa_server *s = new cpaa_server();
    s->posteriori = o.stop_rule == CPAA_STOP_POSTERIORI;
    s->fused = (o.flags & CPAA_SERVER_FUSED) != 0;
    s->frontier = !s->fused && (o.flags & CPAA_SPARSE_FRONTIER) != 0;
    s->budget = device_mem_budget;
    s->prec = o.precision;
    s->normalize = o.normalize;
    s->max_rounds = o.max_rounds > 0 ? o.max_rounds : kDefaultMaxRounds;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && s->fused) e = cudaStreamCreateWithFlags(&s->fstream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
        delete s;
        return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    s->sched = std::thread(scheduler_main, s);
    s->comp_th = std::thread(completion_main, s);
    *out = s;
    return CPAA_OK;
}

extern "C" cpaa_status cpaa_server_add_graph(cpaa_server *s, cpaa_graph *g, int max_slots, int *graph_id) {
    clear_error();
    if (!s || !g || !graph_id) return fail(CPAA_EINVAL, "NULL argument");
    if (max_slots < 0 || max_slots > kMaxWidth) return fail(CPAA_EINVAL, "max_slots must lie in [0, 16]");
    int W = max_slots == 0 ? kMaxWidth : max_slots;
    while (W & (W - 1)) --W;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        while (W >= 1 && s->used + graph_bytes(g, s->prec, W, s->posteriori, s->frontier) > s->budget) W /= 2;
        if (W < 1) return fail(CPAA_ENOMEM, "device memory budget too small for one slot of this graph");
    }
    auto gs = std::make_unique<GraphState>();
    gs->g = g;
    gs->W = W;
    const int64_t n = g->n;
    cpaa_status st = CPAA_OK;
    cudaSetDevice(s->device);
#define SALLOC(ptr, bytes)                                                       \
    do {                                                                         \
        cudaError_t e_ = cudaMalloc((void **)&(ptr), (bytes));                   \
        if (e_ != cudaSuccess) { st = cuda_fail(e_, "cudaMalloc (server slots)"); goto fail_out; } \
    } while (0)
#define SCK(call)                                                                \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) { st = cuda_fail(e_, #call); goto fail_out; }     \
    } while (0)
    {
        const size_t tb = tile_bytes(g, s->prec, W);
        if (s->fused) {  // every graph's work goes to the server's stream
            gs->stream = s->fstream;
            gs->own_stream = false;
        } else {
            SCK(cudaStreamCreateWithFlags(&gs->stream, cudaStreamNonBlocking));
        }
        SALLOC(gs->y[0], tb);
        SALLOC(gs->y[1], tb);
        SALLOC(gs->rho, tb);
        SALLOC(gs->comp, tb);
        SALLOC(gs->spare, tb);
        SALLOC(gs->long_part, (size_t)std::max(1, g->num_hub_tiles) * W * 8);
        SALLOC(gs->long_cnt, (size_t)std::max(1, g->n_hub) * 4);
        SALLOC(gs->red, 2 * 8 * (size_t)W);
        SALLOC(gs->result, (size_t)n * W * 8);
        SALLOC(gs->part, (size_t)kPrepBlocks * 8);
        SALLOC(gs->sums, (size_t)W * 8);
        SCK(cudaMemsetAsync(gs->y[0], 0, tb, gs->stream));
        SCK(cudaMemsetAsync(gs->y[1], 0, tb, gs->stream));
        SCK(cudaMemsetAsync(gs->long_cnt, 0, (size_t)std::max(1, g->n_hub) * 4, gs->stream));
        if (s->posteriori) {
            SALLOC(gs->ipart, 2 * 8 * (size_t)W * ((size_t)g->n_hub + g->num_chunks));
            SALLOC(gs->ipart2, 2 * 8 * (size_t)W * kSumBlocks);
            SALLOC(gs->dstop, sizeof(DevStop));
            SCK(cudaMemsetAsync(gs->dstop, 0, sizeof(DevStop), gs->stream));
            SCK(cudaHostAlloc((void **)&gs->h_ring, sizeof(DevStop) * kInFlight, cudaHostAllocMapped));
            SCK(cudaHostAlloc((void **)&gs->h_slot, sizeof(DevStop) * W, cudaHostAllocMapped));
            SCK(cudaHostGetDevicePointer((void **)&gs->d_ring, gs->h_ring, 0));
            SCK(cudaHostGetDevicePointer((void **)&gs->d_slot, gs->h_slot, 0));
        }
        if (s->frontier && g->nnz >= kFrontierMinEntries) {
            if ((st = ensure_frontier(g, gs->fr, nullptr)) != CPAA_OK) goto fail_out;
            gs->fr_ok = true;
        }
        for (auto &e : gs->ring) SCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        gs->slots.resize(W);
        for (auto &sl : gs->slots) SCK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
        // host copies for admission: caller id -> new id, and degrees
        std::vector<int32_t> perm((size_t)n);
        std::vector<double> deg((size_t)n);
        SCK(cudaMemcpy(perm.data(), g->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        SCK(cudaMemcpy(deg.data(), g->deg64, sizeof(double) * n, cudaMemcpyDeviceToHost));
        gs->inv_perm.resize((size_t)n);
        gs->deg.resize((size_t)n);
        for (int64_t r = 0; r < n; ++r) {
            gs->inv_perm[perm[r]] = (int32_t)r;
            gs->deg[perm[r]] = deg[r];
        }
        SCK(cudaStreamSynchronize(gs->stream));
        gs->bytes = graph_bytes(g, s->prec, W, s->posteriori, s->frontier);
        std::lock_guard<std::mutex> lk(s->mu);
        gs->id = (int)s->graphs.size();
        s->used += gs->bytes;
        *graph_id = gs->id;
        s->graphs.push_back(std::move(gs));
        return CPAA_OK;
    }
fail_out:
    free_graph_state(*gs);
    return st;
#undef SALLOC
#undef SCK
}

extern "C" cpaa_status cpaa_server_submit(cpaa_server *s, int graph_id, int nseeds, const int32_t *seeds,
                                          const double *weights, double c, double tol, uint64_t *ticket) {
    clear_error();
    if (!s || !seeds || !ticket) return fail(CPAA_EINVAL, "NULL argument");
    GraphState *gs = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (graph_id < 0 || graph_id >= (int)s->graphs.size()) return fail(CPAA_ENOTFOUND, "unknown graph id");
        gs = s->graphs[graph_id].get();
    }
    if (nseeds < 1 || nseeds > CPAA_SERVER_MAX_SEEDS)
        return fail(CPAA_EINVAL, "nseeds must lie in [1, CPAA_SERVER_MAX_SEEDS]");
    if (!(c > 0.0 && c < 1.0)) return fail(CPAA_EINVAL, "damping c must lie in (0, 1)");
    if (!(tol > 0.0)) return fail(CPAA_EINVAL, "tol must be > 0");
    const int64_t n = gs->g->n;
    auto r = std::make_shared<Request>();
    r->graph = graph_id;
    r->c = c;
    r->tol = tol;
    r->seeds.count = nseeds;
    double sumw = 0.0, q = 0.0;
    for (int i = 0; i < nseeds; ++i) {
        const int32_t v = seeds[i];
        if (v < 0 || v >= n) return fail(CPAA_EINVAL, "seed vertex out of range");
        for (int j = 0; j < i; ++j)
            if (seeds[j] == v) return fail(CPAA_EINVAL, "seed vertices must be distinct");
        const double w = weights ? weights[i] : 1.0 / nseeds;
        if (!(w >= 0.0) || !(w < INFINITY)) return fail(CPAA_EINVAL, "weights must be finite and >= 0");
        r->seeds.r[i] = gs->inv_perm[v];
        r->seeds.w[i] = w;
        sumw += w;
        q += w * w / gs->deg[v];
    }
    if (!(std::fabs(sumw - 1.0) <= 1e-9)) return fail(CPAA_EINVAL, "weights must sum to 1");
    r->seeds.l1 = sumw;
    r->kappa = std::sqrt((double)gs->g->nnz) * std::sqrt(q);
    r->M = cpaa_rounds_needed(c, tol, r->kappa, s->normalize, s->max_rounds);
    if (r->M < 0) {
        r->M = s->max_rounds;
        r->notconv = true;
    }
    r->t_submit = clk::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (gs->pending.size() >= kMaxQueue) return fail(CPAA_EBUSY, "queue full");
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    gs->pending.push_back(r);
    ++s->submitted;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return CPAA_OK;
}

extern "C" cpaa_status cpaa_server_wait(cpaa_server *s, uint64_t ticket, double *pi, cpaa_info *info,
                                        int64_t timeout_us) {
    clear_error();
    if (!s) return fail(CPAA_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(CPAA_ENOTFOUND, "unknown ticket");
    ReqP r = it->second;
    auto ready = [&]() {
        return (r->state == Request::DONE && !r->collecting && !r->spilling) ||
               r->state == Request::CANCELLED;
    };
    if (timeout_us < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
        return fail(CPAA_ETIMEOUT, "query not finished yet");
    if (r->state == Request::CANCELLED) {
        s->reqs.erase(r->ticket);
        return fail(CPAA_ECANCELLED, "query was cancelled");
    }
    r->collecting = true;  // the slot stays READY until the copy is done
    GraphState *gs = r->gs;
    const int slot = r->slot;
    lk.unlock();
    cudaError_t e = cudaSuccess;
    if (pi) {
        std::lock_guard<std::mutex> ck(s->copy_mu);
        if (gs) {  // still in its slot
            const int64_t n = gs->g->n;
            e = cudaMemcpyAsync(pi, gs->result + (size_t)slot * n, sizeof(double) * n, cudaMemcpyDefault,
                                s->copy_stream);
        } else {   // spilled to host memory
            e = cudaMemcpyAsync(pi, r->host.data(), sizeof(double) * r->host.size(), cudaMemcpyDefault,
                                s->copy_stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
    }
    lk.lock();
    release_slot(s, *r);
    s->reqs.erase(r->ticket);
    lk.unlock();
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (server result)");
    if (info) {
        info->rounds = r->M;
        info->kappa = r->kappa;
        info->bound = r->by_posteriori ? cpaa_l1_bound(r->c, r->M, 2.0 * r->maxl1, s->normalize)
                                       : cpaa_l1_bound(r->c, r->M, r->kappa, s->normalize);
        info->mass = info->l1 = info->sum_pibar = std::numeric_limits<double>::quiet_NaN();  // not reduced when serving
        info->rounds_ms = 0.0;
    }
    if (r->notconv) return fail(CPAA_ENOTCONV, "the L1 bound needs more than max_rounds rounds");
    return CPAA_OK;
}

extern "C" cpaa_status cpaa_server_cancel(cpaa_server *s, uint64_t ticket) {
    clear_error();
    if (!s) return fail(CPAA_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(CPAA_ENOTFOUND, "unknown ticket");
    ReqP r = it->second;
    if (r->state == Request::CANCELLED) return fail(CPAA_EINVAL, "query already cancelled");
    if (r->state == Request::DONE) {
        if (r->collecting || r->spilling) return fail(CPAA_EBUSY, "query result is being copied; retry");
        release_slot(s, *r);  // discard a finished result
        r->state = Request::CANCELLED;
        ++s->cancelled;
        s->cv_done.notify_all();
        return CPAA_OK;
    }
    if (r->state == Request::PENDING) {  // still queued: leave the queue now
        auto &q = s->graphs[r->graph]->pending;
        q.erase(std::remove(q.begin(), q.end(), r), q.end());
        r->state = Request::CANCELLED;
        r->t_done = clk::now();
        ++s->cancelled;
        s->cv_done.notify_all();
        return CPAA_OK;
    }
    r->cancel = true;  // running: the scheduler frees its slot at its next pass
    s->cv_work.notify_one();
    return CPAA_OK;
}

extern "C" cpaa_status cpaa_server_get_stats(cpaa_server *s, cpaa_server_stats *out) {
    clear_error();
    if (!s || !out) return fail(CPAA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->cancelled = s->cancelled;
    out->failed = s->failed;
    out->pending = 0;
    out->running = 0;
    out->slots = 0;
    for (auto &g : s->graphs) {
        out->pending += (int64_t)g->pending.size();
        out->slots += g->W;
        for (auto &sl : g->slots)
            if (sl.st != FREE) ++out->running;
    }
    out->device_bytes = (int64_t)s->used;
    out->p50_us = percentile(s->lat_us, 0.50);
    out->p99_us = percentile(s->lat_us, 0.99);
    double m = 0;
    for (double v : s->lat_us) m += v;
    out->mean_us = s->lat_us.empty() ? 0.0 : m / s->lat_us.size();
    out->admit_p50_us = percentile(s->admit_us, 0.50);
    out->rounds = s->rounds;
    out->round_columns = s->round_columns;
    out->relayouts = s->relayouts;
    return CPAA_OK;
}

extern "C" cpaa_status cpaa_server_destroy(cpaa_server *s) {
    clear_error();
    if (!s) return CPAA_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_comp.notify_all();
    if (s->sched.joinable()) s->sched.join();
    if (s->comp_th.joinable()) s->comp_th.join();
    cudaSetDevice(s->device);
    for (auto &g : s->graphs) cudaStreamSynchronize(g->stream);
    {
        // queries still queued or running end as cancelled
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &kv : s->reqs) kv.second->state = Request::CANCELLED;
        s->cv_done.notify_all();
    }
    for (auto &g : s->graphs) free_graph_state(*g);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->fstream) cudaStreamDestroy(s->fstream);
    delete s;
    return CPAA_OK;
}
