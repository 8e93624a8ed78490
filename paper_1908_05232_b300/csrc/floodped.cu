// floodped.cu -- host side of the C ABI declared in include/floodped.h.
//
// Owns the device memory of one simulation, builds the navigation fields
// (Section 2.1: navigation agents pointing pedestrians toward the exit, the
// sandbag storage and the barrier) with a breadth-first search, and enqueues
// coupled steps.  A step is
// five kernels on two streams:
//     hash_count --+--> scan -> gather -> ped_step (stream 1) --+--> next step
//                  +--> flood (stream 2)                      --+
// Both branches read the state at step n, so they overlap.  ped_step hashes the
// records it writes for step n + 1, which then opens with step_begin (sandbag
// layers and bag snapshot) in place of hash_count where a barrier can be
// built, and with the scan itself elsewhere.  Runs of 64 steps are
// captured once into a CUDA graph per starting clock slot and hash state, and
// replayed.
// The other step mode runs up to 256 steps per launch of the persistent kernel
// (persist.cu).
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "floodped.h"
#include "fp_common.cuh"

namespace {

constexpr int kGraphSteps = 64;
constexpr int kPersistSteps = 256;  // steps per launch of a persistent kernel
constexpr int kProfEvents = 6;  // CUDA events per profiled step
std::string g_create_error;

// 4-connected breadth-first distance over walkable cells from the goal set;
// each reachable cell gets the code (0..7 = E, N, W, S, NE, NW, SW, SE) of the
// neighbour with the strictly smallest distance, earliest in that order on
// ties, diagonals only past two walkable side cells; goal cells get 8 and
// unreachable cells 255.
void build_nav(int nx, int ny, const std::vector<uint8_t> &walk, const std::vector<uint8_t> &goal,
               std::vector<uint8_t> &code) {
    static const int ox[8] = {1, 0, -1, 0, 1, -1, -1, 1};
    static const int oy[8] = {0, 1, 0, -1, 1, 1, -1, -1};
    const size_t n = (size_t)nx * ny;
    std::vector<int> dist(n, -1), frontier;
    frontier.reserve(n);
    for (size_t c = 0; c < n; ++c)
        if (goal[c]) { dist[c] = 0; frontier.push_back((int)c); }
    for (size_t head = 0; head < frontier.size(); ++head) {
        const int c = frontier[head], i = c % nx, j = c / nx;
        for (int k = 0; k < 4; ++k) {
            const int a = i + ox[k], b = j + oy[k];
            if (a < 0 || b < 0 || a >= nx || b >= ny) continue;
            const int d = b * nx + a;
            if (walk[d] && dist[d] < 0) { dist[d] = dist[c] + 1; frontier.push_back(d); }
        }
    }
    code.assign(n, 255);
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            const int c = j * nx + i;
            if (goal[c]) { code[c] = 8; continue; }
            if (dist[c] < 0) continue;
            int best = -1, bestd = dist[c];
            for (int k = 0; k < 8; ++k) {
                const int a = i + ox[k], b = j + oy[k];
                if (a < 0 || b < 0 || a >= nx || b >= ny) continue;
                const int d = dist[b * nx + a];
                if (d < 0) continue;
                if (k >= 4 && (!walk[j * nx + a] || !walk[b * nx + i])) continue;
                if (d < bestd) { bestd = d; best = k; }
            }
            if (best >= 0) code[c] = (uint8_t)best;
        }
    }
}

}  // namespace

struct fp_sim {
    fp_config cfg{};
    FpSim S{};
    int device = 0;
    cudaStream_t stream = nullptr, stream2 = nullptr;
    bool own_stream = true;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int par = 0, slot = 0;
    bool need_prepare = true, pending_time = false;
    // the records of B are already hashed for the next step (bin counts and the
    // evacuee counts of parity par), by the last pedestrian step
    bool hashed = false;
    bool hash_ahead = true;  // ped_step hashes its output records (fp_set_hash_ahead)
    int nb_known = -1;       // the record count of B while the host knows it (since a clear or an add), else -1
    int ids_known = -1;      // the ids issued, likewise
    long long pend_t = 0, pend_step = 0;
    int tile_rows = 16;
    int ped_lanes = 8;   // lanes per pedestrian in the per-step kernel (1, 2, 4, 8, 16)
    // graphs of 64 steps by starting clock slot, whose first step hashes the
    // records of B itself ([0]) or finds them hashed ([1])
    cudaGraphExec_t graphs[2][4] = {};
    std::string err;
    std::vector<void *> allocs;
    std::vector<uint8_t> walk_h, exit_h, bc_h[4];
    std::vector<int> depot_h, barrier_h;
    std::vector<int> door_cells_h, door_of_h;  // entrance doors: cell, door of the cell
    uint4 *read_buf = nullptr;
    bool profiling = false;
    int mode = FP_MODE_KERNELS;
    int persist_ctas = 0;
    unsigned *grid_bar = nullptr;
    std::vector<cudaEvent_t> prof_ev;  // kProfEvents per profiled step
    // surrogate window buffers (allocated by the first fp_surrogate_advance)
    struct Window {
        bool ready = false;
        int tiles_x = 0, tiles_y = 0, ftiles = 0;
        float *u0[3] = {};                  // start state h, hu, hv (padded planes)
        float *fb[2][3] = {};               // plain fallback state by parity
        unsigned short *fb_occ = nullptr;   // evacuees per cell for the fallback
        FpClock *clock = nullptr;           // fallback clock ring; the start clock at the window's slot
        double *bflux = nullptr;            // fallback boundary volumes (discarded)
        unsigned char *wet = nullptr, *fail = nullptr, *flag = nullptr, *mask = nullptr, *keep = nullptr;
        int *list = nullptr, *batch_of = nullptr, *count = nullptr;  // count[0] net tiles, count[1] failed
        float *resid = nullptr;
        unsigned *maxdiff = nullptr;
        void *x16 = nullptr;                // net input: tiles of 266 x 266 pixels, 16 BF16 channels
        float *dU = nullptr;                // net output [tiles][256][256][3]
        cudaStream_t net_stream = nullptr;  // the net runs here, beside the window's pedestrian steps
        cudaEvent_t ev_start = nullptr, ev_input = nullptr, ev_net = nullptr;
        long long done = 0;                 // windows advanced (check cadence)
        int suspend = 0;                    // windows left on the plain update
    } win;
    // steps, hash ms, flood ms, pedestrian chain ms, step ms, cell updates the flood kernel computed,
    // pedestrian kernel ms
    double prof[7] = {0, 0, 0, 0, 0, 0, 0};
    unsigned *blk_runs = nullptr;  // profiling: flood updates computed per 64 x 8 block

    // Every copy of the library is stream-ordered on the simulation's stream and
    // complete when this returns (a plain cudaMemcpy from pageable memory may
    // return before its DMA lands, unordered with this non-blocking stream).
    cudaError_t copy(void *dst, const void *src, size_t bytes) {
        cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        return e;
    }
    int fail(int code, const std::string &msg) {
        err = msg;
        return code;
    }
    int cuda_fail(cudaError_t e, const char *what) {
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return FP_ECUDA;
    }
    template <class T>
    T *dalloc(size_t count) {
        void *p = nullptr;
        if (cudaMalloc(&p, count * sizeof(T) + 16) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, count * sizeof(T) + 16);
        allocs.push_back(p);
        return static_cast<T *>(p);
    }
    void drop_graphs() {
        for (auto &gs : graphs)
            for (auto &g : gs)
                if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    }
    size_t plane_elems() const { return (size_t)S.px * (size_t)(S.ny + 2); }
    size_t flag_blocks() const {
        return (size_t)((S.nx + FP_TX - 1) / FP_TX) * (size_t)((S.ny + FP_BLK_ROWS - 1) / FP_BLK_ROWS);
    }
    size_t muscl_tiles() const { return (size_t)((S.nx + 31) / 32) * (size_t)((S.ny + 7) / 8); }
    // every block "maybe wet": after any write of the water state from outside
    // the flood update, the next two updates run every tile
    cudaError_t reset_water_flags() {
        cudaError_t e = cudaSuccess;
        for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = cudaMemsetAsync(S.blk_wet[p], 1, flag_blocks(), stream);
        for (int p = 0; p < 3 && e == cudaSuccess && S.mflag[0]; ++p)
            e = cudaMemsetAsync(S.mflag[p], 1, muscl_tiles(), stream);
        return e;
    }
};

static int upload_nav(fp_sim *s) {
    const int nx = s->S.nx, ny = s->S.ny;
    const size_t n = (size_t)nx * ny;
    std::vector<uint8_t> goal(n), code, arrive(n);
    for (int g = 0; g < 3; ++g) {
        std::fill(goal.begin(), goal.end(), 0);
        if (g == 0) {
            for (size_t c = 0; c < n; ++c) goal[c] = s->exit_h[c] ? 1 : 0;
        } else {
            const std::vector<int> &cells = g == 1 ? s->depot_h : s->barrier_h;
            for (int c : cells) goal[c] = 1;
        }
        build_nav(nx, ny, s->walk_h, goal, code);
        cudaError_t e = s->copy(const_cast<unsigned char *>(s->S.nav[g]), code.data(), n);
        if (e != cudaSuccess) return s->cuda_fail(e, "nav upload");
        // the cell the code points to is a goal cell: one load beside the code on the device
        static const int ox[8] = {1, 0, -1, 0, 1, -1, -1, 1};
        static const int oy[8] = {0, 1, 0, -1, 1, 1, -1, -1};
        for (size_t c = 0; c < n; ++c) {
            if (code[c] >= 8) continue;
            const int i = (int)(c % nx) + ox[code[c]], j = (int)(c / nx) + oy[code[c]];
            if (code[(size_t)j * nx + i] == FP_AT_GOAL) arrive[c] |= (uint8_t)(1u << g);
        }
    }
    cudaError_t e = s->copy(const_cast<unsigned char *>(s->S.arrive), arrive.data(), n);
    if (e != cudaSuccess) return s->cuda_fail(e, "nav upload");
    return FP_OK;
}

static void update_inflow_flag(fp_sim *s) {
    int f = 0, nd = 0;
    for (int e = 0; e < 4; ++e)
        for (uint8_t c : s->bc_h[e]) {
            f |= (c == FP_BC_INFLOW);
            nd += (c == FP_BC_DISCHARGE);
        }
    s->S.has_inflow = f;
    // the breach width B: the discharge cells' total length, from the FP32 cell side
    s->S.q_width = (double)nd * (double)s->S.dx;
    s->S.has_discharge = (nd > 0 && s->S.n_q > 0) ? 1 : 0;
}

// copy a caller grid (host or device) into a padded device plane
static cudaError_t put_plane(fp_sim *s, float *dst, const float *src) {
    const FpSim &S = s->S;
    return cudaMemcpy2DAsync(dst + S.px + FP_PADX, (size_t)S.px * 4, src, (size_t)S.nx * 4, (size_t)S.nx * 4, S.ny,
                             cudaMemcpyDefault, s->stream);
}

static cudaError_t get_plane(fp_sim *s, void *dst, const float *src) {
    const FpSim &S = s->S;
    return cudaMemcpy2DAsync(dst, (size_t)S.nx * 4, src + S.px + FP_PADX, (size_t)S.px * 4, (size_t)S.nx * 4, S.ny,
                             cudaMemcpyDefault, s->stream);
}

// Undo a hash of B made ahead by the last pedestrian step (zero the bin counts
// and the evacuee counts of parity par), before anything that rewrites B,
// hashes it by itself or changes the parity.
static cudaError_t drop_hash(fp_sim *s) {
    if (!s->hashed) return cudaSuccess;
    s->hashed = false;
    cudaError_t e = cudaMemsetAsync(s->S.bin_count, 0, ((size_t)s->S.nbins + 1) * sizeof(int), s->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->S.tile_sum, 0, (size_t)fp_scan_tiles(s->S.nbins) * sizeof(int), s->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->S.occ[s->par], 0, s->plane_elems() * sizeof(unsigned short), s->stream);
    return e;
}

// Before the next step after a change from outside: the clock ring, the water
// flags and the clock's wave speed, all ordered on the simulation's stream (no
// wait for the work enqueued here; the clock read, when no time was set, is a
// stream-ordered copy).
static int prepare(fp_sim *s) {
    cudaError_t e = drop_hash(s);
    if (e != cudaSuccess) return s->cuda_fail(e, "prepare hash");
    FpClock ring[4];
    memset(ring, 0, sizeof(ring));
    if (s->pending_time) {
        ring[s->slot].t = s->pend_t;
        ring[s->slot].step = s->pend_step;
        s->pending_time = false;
    } else {
        FpClock cur;
        e = s->copy(&cur, &s->S.clock[s->slot], sizeof(cur));
        if (e != cudaSuccess) return s->cuda_fail(e, "clock read");
        ring[s->slot].t = cur.t;
        ring[s->slot].step = cur.step;
    }
    e = cudaMemcpyAsync(s->S.clock, ring, sizeof(ring), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "clock write");
    e = s->reset_water_flags();
    if (e == cudaSuccess) e = cudaMemsetAsync(&s->S.cnt->flood_ticket, 0, sizeof(unsigned), s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "water flags");
    fp_launch_init_clock(s->S, s->par, s->slot, s->stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return s->cuda_fail(e, "prepare");
    s->need_prepare = false;
    return FP_OK;
}

// One coupled step.  ev (profiling only): kProfEvents events -- before
// hash_count (or step_begin), after it, after the flood kernel (stream 2),
// after the pedestrian chain (stream 1), before the flood kernel (stream 2),
// before the pedestrian kernel (stream 1).  The pedestrian kernel hashes its output records
// for the next step, which then opens with step_begin alone.
static void launch_step(fp_sim *s, int par, int slot, cudaEvent_t *ev = nullptr) {
    const FpSim &S = s->S;
    if (ev) cudaEventRecordWithFlags(ev[0], s->stream, cudaEventRecordExternal);
    // With the records hashed ahead, a step opens with step_begin only where a
    // barrier can be built (sandbag layers, bag snapshot); the scan clears the
    // histogram.
    const bool opening = !s->hashed || (S.nb > 0 && S.n_layers > 0);
    if (!s->hashed) fp_launch_hash_count(S, par, s->stream);
    else if (opening) fp_launch_step_begin(S, s->stream);
    cudaEventRecord(s->ev_fork, s->stream);
    if (ev) cudaEventRecordWithFlags(ev[1], s->stream, cudaEventRecordExternal);
    cudaStreamWaitEvent(s->stream2, s->ev_fork, 0);
    // the flood update on stream 2; the pedestrian chain, the longer branch, on
    // stream 1 with programmatic dependent launches on its kernel -> kernel
    // edges (not in profiling mode, whose events sit between the kernels)
    const bool pdl = ev == nullptr;
    if (ev) cudaEventRecordWithFlags(ev[4], s->stream2, cudaEventRecordExternal);
    if (S.order == 2) fp_launch_muscl(S, par, slot, s->stream2);
    else fp_launch_flood(S, par, slot, s->tile_rows, s->stream2);
    if (ev) cudaEventRecordWithFlags(ev[2], s->stream2, cudaEventRecordExternal);
    fp_launch_scan(S, s->stream, pdl);
    fp_launch_gather(S, slot, s->stream, pdl);
    if (ev) cudaEventRecordWithFlags(ev[5], s->stream, cudaEventRecordExternal);
    fp_launch_ped_step(S, par, slot, s->ped_lanes, s->stream, pdl, s->hash_ahead);
    if (ev) cudaEventRecordWithFlags(ev[3], s->stream, cudaEventRecordExternal);
    cudaEventRecord(s->ev_join, s->stream2);
    cudaStreamWaitEvent(s->stream, s->ev_join, 0);
    s->hashed = s->hash_ahead;
}

// A coupled step whose flood update moves no water (surrogate window): the
// pedestrian chain as in launch_step (here on stream 2); on stream 1 only the
// clock advance and the clearing of the evacuee counts the flood kernel would
// have consumed.
// Both parities of the state must hold the same water state.
static void launch_window_step(fp_sim *s, int par, int slot) {
    const FpSim &S = s->S;
    fp_launch_hash_count(S, par, s->stream);
    cudaEventRecord(s->ev_fork, s->stream);
    cudaStreamWaitEvent(s->stream2, s->ev_fork, 0);
    fp_launch_clock_advance(S, slot, s->stream);
    cudaMemsetAsync(S.occ[par], 0, s->plane_elems() * sizeof(unsigned short), s->stream);
    fp_launch_scan(S, s->stream2);
    fp_launch_gather(S, slot, s->stream2);
    fp_launch_ped_step(S, par, slot, s->ped_lanes, s->stream2);
    cudaEventRecord(s->ev_join, s->stream2);
    cudaStreamWaitEvent(s->stream, s->ev_join, 0);
}

static int ensure_window(fp_sim *s) {
    fp_sim::Window &W = s->win;
    if (W.ready) return FP_OK;
    const FpSim &S = s->S;
    W.tiles_x = (S.nx + FP_SUR_TILE - 1) / FP_SUR_TILE;
    W.tiles_y = (S.ny + FP_SUR_TILE - 1) / FP_SUR_TILE;
    const int nt = W.tiles_x * W.tiles_y;
    W.ftiles = ((S.nx + FP_TX - 1) / FP_TX) * ((S.ny + s->tile_rows - 1) / s->tile_rows);
    const size_t pe = s->plane_elems();
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        ok &= (W.u0[k] = s->dalloc<float>(pe)) != nullptr;
        ok &= (W.fb[0][k] = s->dalloc<float>(pe)) != nullptr;
        ok &= (W.fb[1][k] = s->dalloc<float>(pe)) != nullptr;
    }
    ok &= (W.fb_occ = s->dalloc<unsigned short>(pe + 2)) != nullptr;
    ok &= (W.clock = s->dalloc<FpClock>(4)) != nullptr;
    ok &= (W.bflux = s->dalloc<double>(2 * (size_t)S.nx + 2 * (size_t)S.ny)) != nullptr;
    ok &= (W.wet = s->dalloc<unsigned char>(nt)) != nullptr;
    ok &= (W.fail = s->dalloc<unsigned char>(nt)) != nullptr;
    ok &= (W.flag = s->dalloc<unsigned char>(nt)) != nullptr;
    ok &= (W.keep = s->dalloc<unsigned char>(nt)) != nullptr;
    ok &= (W.mask = s->dalloc<unsigned char>(W.ftiles)) != nullptr;
    ok &= (W.list = s->dalloc<int>(nt)) != nullptr;
    ok &= (W.batch_of = s->dalloc<int>(nt)) != nullptr;
    ok &= (W.count = s->dalloc<int>(2)) != nullptr;
    ok &= (W.resid = s->dalloc<float>(nt)) != nullptr;
    ok &= (W.maxdiff = s->dalloc<unsigned>(1)) != nullptr;
    ok &= (W.x16 = s->dalloc<unsigned char>((size_t)nt * (FP_SUR_TILE + 2 * FP_SUR_HALO) *
                                            fp_sur_pitch(FP_SUR_TILE + 2 * FP_SUR_HALO) * 32)) != nullptr;
    ok &= (W.dU = s->dalloc<float>((size_t)nt * FP_SUR_TILE * FP_SUR_TILE * 3)) != nullptr;
    if (!ok) return s->fail(FP_ENOMEM, "surrogate window buffers");
    if (cudaStreamCreateWithFlags(&W.net_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&W.ev_start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&W.ev_input, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&W.ev_net, cudaEventDisableTiming) != cudaSuccess)
        return s->fail(FP_ECUDA, "surrogate window stream");
    W.ready = true;
    return FP_OK;
}

// Persistent kernel with the global timer stamped by CTA 0 at every phase end.
static int step_profiled_persistent(fp_sim *s, int n) {
    const cudaError_t eh = drop_hash(s);  // the persistent kernel hashes B itself
    if (eh != cudaSuccess) return s->cuda_fail(eh, "hash reset");
    int left = n;
    while (left > 0) {
        const int m = left < 256 ? left : 256;
        const size_t cnt = 4 * (size_t)m + 1;
        unsigned long long *ts = s->dalloc<unsigned long long>(cnt);
        if (!ts) return s->fail(FP_ENOMEM, "profile stamps");
        FpSim S = s->S;
        S.phase_ts = ts;
        S.phase_ts_steps = m;
        cudaError_t e = fp_launch_persistent(S, s->par, s->slot, m, s->grid_bar, s->persist_ctas, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        std::vector<unsigned long long> h(cnt);
        if (e == cudaSuccess) e = s->copy(h.data(), ts, cnt * sizeof(unsigned long long));
        s->allocs.pop_back();
        cudaFree(ts);
        if (e != cudaSuccess) return s->cuda_fail(e, "profiled persistent steps");
        for (int k = 0; k < m; ++k) {
            const double a = (double)(h[4 * k + 1] - h[4 * k]) * 1e-6;      // scan phase
            const double b = (double)(h[4 * k + 2] - h[4 * k + 1]) * 1e-6;  // prefix + gather
            const double c = (double)(h[4 * k + 4] - h[4 * k + 2]) * 1e-6;  // flood + pedestrians
            s->prof[0] += 1;
            s->prof[1] += a;
            s->prof[2] += c;
            s->prof[3] += b;
            s->prof[4] += a + b + c;
        }
        if (m & 1) s->par ^= 1;
        s->slot = (s->slot + m) & 3;
        left -= m;
    }
    return FP_OK;
}

// Cell updates the flood kernel computed (tiles not skipped as dry) since
// profiling was switched on.
static int count_computed_cells(fp_sim *s) {
    const FpSim &S = s->S;
    const int bw = (S.nx + FP_TX - 1) / FP_TX, bh = (S.ny + FP_BLK_ROWS - 1) / FP_BLK_ROWS;
    std::vector<unsigned> runs((size_t)bw * bh);
    const cudaError_t e = s->copy(runs.data(), s->blk_runs, runs.size() * sizeof(unsigned));
    if (e != cudaSuccess) return s->cuda_fail(e, "profile block counts");
    double cells = 0.0;
    for (int r = 0; r < bh; ++r)
        for (int c = 0; c < bw; ++c)
            cells += (double)runs[(size_t)r * bw + c] * std::min(FP_TX, S.nx - c * FP_TX) *
                     std::min(FP_BLK_ROWS, S.ny - r * FP_BLK_ROWS);
    s->prof[5] = cells;
    return FP_OK;
}

static int step_profiled_kernels(fp_sim *s, int n);

static int step_profiled(fp_sim *s, int n) {
    const int rc = s->mode == FP_MODE_PERSISTENT ? step_profiled_persistent(s, n) : step_profiled_kernels(s, n);
    return rc != FP_OK ? rc : count_computed_cells(s);
}

static int step_profiled_kernels(fp_sim *s, int n) {
    if ((int)s->prof_ev.size() < kProfEvents * n) {
        for (int k = (int)s->prof_ev.size(); k < kProfEvents * n; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return s->fail(FP_ECUDA, "event create");
            s->prof_ev.push_back(e);
        }
    }
    // The steps and their events are captured into one graph and replayed, as
    // in the timed runs: launched one by one from the host, a slow host would
    // leave gaps between the kernels that the events would count.
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return s->cuda_fail(e, "profiled capture");
    for (int k = 0; k < n; ++k) {
        launch_step(s, s->par, s->slot, &s->prof_ev[kProfEvents * k]);
        s->par ^= 1;
        s->slot = (s->slot + 1) & 3;
    }
    e = cudaStreamEndCapture(s->stream, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return s->cuda_fail(e, "profiled steps");
    for (int k = 0; k < n; ++k) {
        cudaEvent_t *ev = &s->prof_ev[kProfEvents * k];
        float a = 0, b = 0, c = 0, d = 0, f = 0;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&b, ev[4], ev[2]);  // the flood kernel, on its own stream
        cudaEventElapsedTime(&c, ev[1], ev[3]);
        cudaEventElapsedTime(&d, ev[0], ev[2]);
        cudaEventElapsedTime(&f, ev[5], ev[3]);  // the pedestrian kernel
        s->prof[6] += f;
        s->prof[0] += 1;
        s->prof[1] += a;
        s->prof[2] += b;
        s->prof[3] += c;
        s->prof[4] += std::max(d, a + c);
    }
    return FP_OK;
}

extern "C" {

int fp_sim_create(const fp_config *cfg, fp_sim **out) {
    if (!cfg || !out) { g_create_error = "null argument"; return FP_EINVAL; }
    *out = nullptr;
    const fp_config &c = *cfg;
    if (c.nx < 1 || c.ny < 1 || c.nx > (1 << 16) || c.ny > (1 << 16) || !(c.dx > 0.0f) || !(c.g > 0.0f) ||
        !(c.cfl > 0.0f) || c.cfl > 1.0f || c.max_peds < 0 || c.max_peds > (1 << 26) || !(c.t_end >= 0.0) ||
        !(c.ped_noise >= 0.0f) ||
        (c.tile_rows != 0 && c.tile_rows != 8 && c.tile_rows != 16 && c.tile_rows != 32) ||
        (c.riemann != FP_RIEMANN_HLL && c.riemann != FP_RIEMANN_HLLC) || c.order < 0 || c.order > 2) {
        g_create_error = "invalid fp_config";
        return FP_EINVAL;
    }
    fp_sim *s = new fp_sim();
    s->cfg = c;
    cudaGetDevice(&s->device);
    FpSim &S = s->S;
    S.nx = c.nx;
    S.ny = c.ny;
    S.px = ((c.nx + 2 * FP_PADX + 7) / 8) * 8;  // >= 4 guard columns each side; 16-byte rows of uint16
    S.dx = c.dx;
    S.g = c.g;
    S.cfl = c.cfl;
    S.ped_noise = c.ped_noise;
    S.t_end = (long long)llround(c.t_end * 1048576.0);
    S.seed = c.seed;
    S.coupling = c.coupling ? 1 : 0;
    S.evac_trigger = c.evac_trigger ? 1 : 0;
    S.cap = c.max_peds;
    S.hk = std::max(1, (int)std::ceil(1.0 / (double)c.dx));
    S.nbx = (c.nx + S.hk - 1) / S.hk;
    S.nby = (c.ny + S.hk - 1) / S.hk;
    S.nbins = S.nbx * S.nby;
    S.bpc = (int)std::ceil(((double)c.dx * (double)c.dx) / (0.40 * 0.30));
    S.barrier_polls = FP_BARRIER_POLLS_DEFAULT;
    S.riemann = c.riemann;
    S.order = c.order == 2 ? 2 : 1;
    s->tile_rows = c.tile_rows ? c.tile_rows : 16;
    const size_t pe = s->plane_elems(), n = (size_t)c.nx * c.ny;
    bool ok = true;
    for (int p = 0; p < 2; ++p) {
        ok &= (S.h[p] = s->dalloc<float>(pe)) != nullptr;
        ok &= (S.hu[p] = s->dalloc<float>(pe)) != nullptr;
        ok &= (S.hv[p] = s->dalloc<float>(pe)) != nullptr;
    }
    ok &= (S.z = s->dalloc<float>(pe)) != nullptr;
    if (S.order == 2) {
        ok &= (S.mh = s->dalloc<float>(pe)) != nullptr;
        ok &= (S.mhu = s->dalloc<float>(pe)) != nullptr;
        ok &= (S.mhv = s->dalloc<float>(pe)) != nullptr;
        for (int p = 0; p < 3; ++p) ok &= (S.mflag[p] = s->dalloc<unsigned char>(s->muscl_tiles())) != nullptr;
    }
    ok &= (S.n0 = s->dalloc<float>(pe)) != nullptr;
    ok &= (S.occ[0] = s->dalloc<unsigned short>(pe + 2)) != nullptr;
    ok &= (S.occ[1] = s->dalloc<unsigned short>(pe + 2)) != nullptr;
    for (int p = 0; p < 2; ++p) ok &= (S.blk_wet[p] = s->dalloc<unsigned char>(s->flag_blocks())) != nullptr;
    unsigned char *bcd[4];
    for (int e = 0; e < 4; ++e) {
        const int len = e < 2 ? c.nx : c.ny;
        ok &= (bcd[e] = s->dalloc<unsigned char>(len)) != nullptr;
        S.bc[e] = bcd[e];
        s->bc_h[e].assign(len, FP_BC_WALL);
    }
    unsigned char *walk = s->dalloc<unsigned char>(n), *arrive = s->dalloc<unsigned char>(n);
    unsigned *nbr = s->dalloc<unsigned>(n);
    ok &= walk && arrive && nbr;
    S.walk = walk;
    S.nbr = nbr;
    S.arrive = arrive;
    for (int g = 0; g < 3; ++g) ok &= (S.nav[g] = s->dalloc<unsigned char>(n)) != nullptr;
    double *ht = s->dalloc<double>(FP_MAX_HYDRO), *hh = s->dalloc<double>(FP_MAX_HYDRO);
    double *qt = s->dalloc<double>(FP_MAX_HYDRO), *qq = s->dalloc<double>(FP_MAX_HYDRO);
    ok &= ht && hh && qt && qq;
    S.hydro_t = ht;
    S.hydro_h = hh;
    S.q_t = qt;
    S.q_Q = qq;
    S.h_qin = 1.0;
    ok &= (S.clock = s->dalloc<FpClock>(4)) != nullptr;
    ok &= (S.cnt = s->dalloc<FpCounters>(1)) != nullptr;
    const size_t cap = (size_t)std::max(1, c.max_peds);
    ok &= (S.pedA = s->dalloc<uint4>(2 * cap)) != nullptr;
    ok &= (S.posA = s->dalloc<float2>(cap)) != nullptr;
    ok &= (S.xiA = s->dalloc<float2>(cap)) != nullptr;
    ok &= (S.pedB = s->dalloc<uint4>(2 * cap)) != nullptr;
    ok &= (S.arch = s->dalloc<uint4>(2 * cap)) != nullptr;
    ok &= (s->read_buf = s->dalloc<uint4>(2 * cap)) != nullptr;
    ok &= (S.bin_count = s->dalloc<int>((size_t)S.nbins + 1)) != nullptr;
    ok &= (S.bin_start = s->dalloc<int>((size_t)S.nbins + 2)) != nullptr;
    ok &= (S.pkey = s->dalloc<int>(cap)) != nullptr;
    ok &= (S.pslot = s->dalloc<int>(cap)) != nullptr;
    ok &= (S.tile_sum = s->dalloc<int>((size_t)fp_scan_tiles(S.nbins))) != nullptr;
    ok &= (S.bflux = s->dalloc<double>(2 * (size_t)c.nx + 2 * (size_t)c.ny)) != nullptr;
    ok &= (S.partials = s->dalloc<double>(148 * 4)) != nullptr;
    ok &= (S.scan_part = s->dalloc<int>(2048)) != nullptr;
    ok &= (s->grid_bar = s->dalloc<unsigned>(4)) != nullptr;  // persistent kernel: barrier word, 2 tickets
    if (!ok) {
        g_create_error = "device allocation failed";
        fp_destroy(s);
        return FP_ENOMEM;
    }
    // defaults: flat dry walkable terrain, n = 0.01, walls, no hydrograph
    s->walk_h.assign(n, 1);
    s->exit_h.assign(n, 0);
    std::vector<float> n0(n, 0.01f);
    cudaMemset(walk, 1, n);
    cudaMemcpy2D(S.n0 + S.px + FP_PADX, (size_t)S.px * 4, n0.data(), (size_t)c.nx * 4, (size_t)c.nx * 4, c.ny,
                 cudaMemcpyHostToDevice);
    cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&s->stream2, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming);
    int rc = upload_nav(s);
    if (rc == FP_OK) {
        cudaError_t ea = fp_flood_init_attributes();
        if (ea != cudaSuccess) rc = s->cuda_fail(ea, "flood kernel attributes");
    }
    if (rc == FP_OK) {
        s->persist_ctas = fp_persistent_ctas();
        cudaGetLastError();
        s->mode = FP_MODE_KERNELS;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (rc == FP_OK && e != cudaSuccess) rc = s->cuda_fail(e, "create");
    if (rc != FP_OK) {
        g_create_error = s->err;
        fp_destroy(s);
        return rc;
    }
    *out = s;
    return FP_OK;
}

int fp_set_stream(fp_sim *s, void *cuda_stream) {
    if (!s) return FP_EINVAL;
    cudaStreamSynchronize(s->stream);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    if (cuda_stream) {
        s->stream = static_cast<cudaStream_t>(cuda_stream);
        s->own_stream = false;
    } else {
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        s->own_stream = true;
    }
    s->drop_graphs();
    return FP_OK;
}

int fp_set_terrain(fp_sim *s, const float *z, const float *n0, const uint8_t *walkable, const uint8_t *exit_mask) {
    if (!s || !z || !n0 || !walkable || !exit_mask) return s ? s->fail(FP_EINVAL, "null terrain array") : FP_EINVAL;
    const size_t n = (size_t)s->S.nx * s->S.ny;
    cudaError_t e;
    if ((e = put_plane(s, s->S.z, z)) != cudaSuccess) return s->cuda_fail(e, "z upload");
    if ((e = put_plane(s, s->S.n0, n0)) != cudaSuccess) return s->cuda_fail(e, "n0 upload");
    if ((e = s->copy(s->walk_h.data(), walkable, n)) != cudaSuccess)
        return s->cuda_fail(e, "walkable copy");
    if ((e = s->copy(s->exit_h.data(), exit_mask, n)) != cudaSuccess)
        return s->cuda_fail(e, "exit copy");
    for (auto &v : s->walk_h) v = v ? 1 : 0;
    {  // device cell flags: bit 0 walkable, bit 1 exit
        std::vector<uint8_t> flags(n);
        for (size_t c = 0; c < n; ++c) flags[c] = (uint8_t)(s->walk_h[c] | (s->exit_h[c] ? 2 : 0));
        if ((e = s->copy(const_cast<unsigned char *>(s->S.walk), flags.data(), n)) != cudaSuccess)
            return s->cuda_fail(e, "walkable upload");
        // the flags of every cell's 3 x 3 neighbourhood in one word (a
        // pedestrian's move mostly ends next to its cell)
        const int nx = s->S.nx, ny = s->S.ny;
        std::vector<unsigned> nb(n, 0u);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                unsigned f = 0u;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int a = i + dx, b = j + dy;
                        if (a >= 0 && b >= 0 && a < nx && b < ny)
                            f |= (unsigned)(flags[(size_t)b * nx + a] & 3u) << (2 * ((dy + 1) * 3 + dx + 1));
                    }
                nb[(size_t)j * nx + i] = f;
            }
        if ((e = s->copy(const_cast<unsigned *>(s->S.nbr), nb.data(), n * sizeof(unsigned))) != cudaSuccess)
            return s->cuda_fail(e, "walkable upload");
    }
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return s->cuda_fail(e, "terrain");
    // the doors' fields follow the old walkability: set them again after the terrain
    s->S.n_doors = 0;
    s->door_cells_h.clear();
    s->door_of_h.clear();
    s->drop_graphs();
    return upload_nav(s);
}

int fp_set_bed(fp_sim *s, const float *z) {
    if (!s) return FP_EINVAL;
    if (!z) return s->fail(FP_EINVAL, "null bed array");
    cudaError_t e = put_plane(s, s->S.z, z);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "z upload");
    s->need_prepare = true;
    return FP_OK;
}

int fp_set_boundary(fp_sim *s, int32_t edge, const uint8_t *codes) {
    if (!s) return FP_EINVAL;
    if (edge < 0 || edge > 3 || !codes) return s->fail(FP_EINVAL, "bad edge or codes");
    const int len = edge < 2 ? s->S.nx : s->S.ny;
    std::vector<uint8_t> h(len);
    cudaError_t e = s->copy(h.data(), codes, len);
    if (e != cudaSuccess) return s->cuda_fail(e, "boundary copy");
    for (uint8_t c : h)
        if (c > FP_BC_DISCHARGE) return s->fail(FP_EINVAL, "boundary code out of range");
    s->bc_h[edge] = h;
    e = s->copy(const_cast<unsigned char *>(s->S.bc[edge]), h.data(), len);
    if (e != cudaSuccess) return s->cuda_fail(e, "boundary upload");
    update_inflow_flag(s);
    s->drop_graphs();
    s->need_prepare = true;  // the clock's inflow speeds
    return FP_OK;
}

int fp_set_discharge(fp_sim *s, const double *t, const double *q, int32_t n, double h_inflow) {
    if (!s) return FP_EINVAL;
    if (!t || !q || n < 1 || n > FP_MAX_HYDRO) return s->fail(FP_EINVAL, "discharge hydrograph needs 1..64 points");
    if (!(h_inflow > 0.0) || !std::isfinite(h_inflow)) return s->fail(FP_EINVAL, "inflow depth must be > 0");
    std::vector<double> th(n), qh(n);
    cudaError_t e = s->copy(th.data(), t, n * sizeof(double));
    if (e == cudaSuccess) e = s->copy(qh.data(), q, n * sizeof(double));
    if (e != cudaSuccess) return s->cuda_fail(e, "discharge copy");
    for (int k = 0; k < n; ++k) {
        if (!(qh[k] >= 0.0) || !std::isfinite(qh[k]) || !std::isfinite(th[k]))
            return s->fail(FP_EINVAL, "discharge values");
        if (k && !(th[k] > th[k - 1])) return s->fail(FP_EINVAL, "discharge times must increase");
    }
    s->copy(const_cast<double *>(s->S.q_t), th.data(), n * sizeof(double));
    e = s->copy(const_cast<double *>(s->S.q_Q), qh.data(), n * sizeof(double));
    if (e != cudaSuccess) return s->cuda_fail(e, "discharge upload");
    s->S.n_q = n;
    s->S.h_qin = (double)(float)h_inflow;
    // Q = 0 from the point after the last positive one on (never, if the table ends positive)
    long long end = 0;
    if (qh[n - 1] > 0.0) {
        end = LLONG_MAX;
    } else {
        for (int k = n - 2; k >= 0; --k)
            if (qh[k] > 0.0) {
                end = (long long)std::ceil(th[k + 1] * 1048576.0);
                break;
            }
    }
    s->S.q_end_ticks = end;
    update_inflow_flag(s);
    s->drop_graphs();
    s->need_prepare = true;
    return FP_OK;
}

int fp_set_hydrograph(fp_sim *s, const double *t, const double *h, int32_t n) {
    if (!s) return FP_EINVAL;
    if (!t || !h || n < 1 || n > FP_MAX_HYDRO) return s->fail(FP_EINVAL, "hydrograph needs 1..64 points");
    std::vector<double> th(n), hh(n);
    s->copy(th.data(), t, n * sizeof(double));
    s->copy(hh.data(), h, n * sizeof(double));
    for (int k = 0; k < n; ++k) {
        if (!(hh[k] >= 0.0) || !std::isfinite(th[k])) return s->fail(FP_EINVAL, "hydrograph values");
        if (k && !(th[k] > th[k - 1])) return s->fail(FP_EINVAL, "hydrograph times must increase");
    }
    s->copy(const_cast<double *>(s->S.hydro_t), th.data(), n * sizeof(double));
    cudaError_t e = s->copy(const_cast<double *>(s->S.hydro_h), hh.data(), n * sizeof(double));
    if (e != cudaSuccess) return s->cuda_fail(e, "hydrograph upload");
    s->S.n_hydro = n;
    s->drop_graphs();
    s->need_prepare = true;
    return FP_OK;
}

int fp_set_doors(fp_sim *s, const int32_t *cells, const int32_t *door, int32_t n_cells, int32_t n_doors,
                 double entry_period_s, double v0_min, double v0_max) {
    if (!s) return FP_EINVAL;
    if (n_doors < 0 || n_doors > FP_MAX_DOORS) return s->fail(FP_EINVAL, "door count out of range");
    cudaError_t e = cudaStreamSynchronize(s->stream);  // no step in flight reads the tables
    if (e != cudaSuccess) return s->cuda_fail(e, "doors");
    if (n_doors == 0) {
        s->S.n_doors = 0;
        s->door_cells_h.clear();
        s->door_of_h.clear();
        s->drop_graphs();
        return FP_OK;
    }
    if (n_cells < n_doors || !cells || !door) return s->fail(FP_EINVAL, "bad door cell arguments");
    if (!(entry_period_s >= 1.0 / 1024.0 && entry_period_s <= 1e9))
        return s->fail(FP_EINVAL, "entry period out of range");
    if (!(v0_min >= 0.0 && v0_max >= v0_min && v0_max <= 10.0)) return s->fail(FP_EINVAL, "bad walking speeds");
    const int nx = s->S.nx, ny = s->S.ny;
    const size_t n = (size_t)nx * ny;
    std::vector<int> hc(n_cells), hd(n_cells);
    if ((e = s->copy(hc.data(), cells, sizeof(int) * n_cells)) != cudaSuccess) return s->cuda_fail(e, "door copy");
    if ((e = s->copy(hd.data(), door, sizeof(int) * n_cells)) != cudaSuccess) return s->cuda_fail(e, "door copy");
    int entry[FP_MAX_DOORS];
    for (int d = 0; d < FP_MAX_DOORS; ++d) entry[d] = -1;
    for (int k = 0; k < n_cells; ++k) {
        if (hc[k] < 0 || (size_t)hc[k] >= n || hd[k] < 0 || hd[k] >= n_doors)
            return s->fail(FP_EINVAL, "door cell or door index out of range");
        if (!s->walk_h[hc[k]]) return s->fail(FP_EINVAL, "a door cell is not walkable");
        if (entry[hd[k]] < 0) entry[hd[k]] = hc[k];
    }
    for (int d = 0; d < n_doors; ++d)
        if (entry[d] < 0) return s->fail(FP_EINVAL, "a door has no cell");
    if (!s->S.door_nav) {
        unsigned char *nav = s->dalloc<unsigned char>((size_t)FP_MAX_DOORS * n), *arr = s->dalloc<unsigned char>(n);
        if (!nav || !arr) return s->fail(FP_ECUDA, "door table allocation failed");
        s->S.door_nav = nav;
        s->S.door_arrive = arr;
    }
    // one navigation field per door (the same breadth-first construction as
    // the exit's) and the arrival bits
    std::vector<uint8_t> goal(n), code, arrive(n, 0);
    static const int ox[8] = {1, 0, -1, 0, 1, -1, -1, 1};
    static const int oy[8] = {0, 1, 0, -1, 1, 1, -1, -1};
    for (int d = 0; d < n_doors; ++d) {
        std::fill(goal.begin(), goal.end(), 0);
        for (int k = 0; k < n_cells; ++k)
            if (hd[k] == d) goal[hc[k]] = 1;
        build_nav(nx, ny, s->walk_h, goal, code);
        e = s->copy(const_cast<unsigned char *>(s->S.door_nav) + (size_t)d * n, code.data(), n);
        if (e != cudaSuccess) return s->cuda_fail(e, "door navigation upload");
        for (size_t c = 0; c < n; ++c) {
            if (code[c] >= 8) continue;
            const int i = (int)(c % nx) + ox[code[c]], j = (int)(c / nx) + oy[code[c]];
            if (code[(size_t)j * nx + i] == FP_AT_GOAL) arrive[c] |= (uint8_t)(1u << d);
        }
    }
    if ((e = s->copy(const_cast<unsigned char *>(s->S.door_arrive), arrive.data(), n)) != cudaSuccess)
        return s->cuda_fail(e, "door navigation upload");
    s->S.n_doors = n_doors;
    for (int d = 0; d < FP_MAX_DOORS; ++d) s->S.door_entry[d] = d < n_doors ? entry[d] : 0;
    s->S.entry_period = std::max(1LL, (long long)llround(entry_period_s * 1048576.0));
    const float lo = (float)v0_min, hi = (float)v0_max;
    s->S.entry_vlo = lo;
    s->S.entry_vspan = hi - lo;  // FP32 difference
    s->door_cells_h = hc;
    s->door_of_h = hd;
    s->drop_graphs();  // the graphs hold the kernels' parameters
    return FP_OK;
}

int fp_set_goals(fp_sim *s, const int32_t *depot, int32_t n_depot, const int32_t *barrier, int32_t n_barrier,
                 int32_t n_layers) {
    if (!s) return FP_EINVAL;
    const int n = s->S.nx * s->S.ny;
    if (n_depot < 0 || n_barrier < 0 || n_layers < 0 || (n_depot && !depot) || (n_barrier && !barrier))
        return s->fail(FP_EINVAL, "bad goal arguments");
    std::vector<int> dh(n_depot), bh(n_barrier);
    if (n_depot) s->copy(dh.data(), depot, n_depot * sizeof(int));
    if (n_barrier) s->copy(bh.data(), barrier, n_barrier * sizeof(int));
    for (int c : dh)
        if (c < 0 || c >= n) return s->fail(FP_EINVAL, "depot cell out of range");
    for (int c : bh)
        if (c < 0 || c >= n) return s->fail(FP_EINVAL, "barrier cell out of range");
    s->depot_h = dh;
    s->barrier_h = bh;
    if (n_barrier) {
        int *d = s->dalloc<int>(n_barrier);
        if (!d) return s->fail(FP_ENOMEM, "barrier allocation");
        s->copy(d, bh.data(), n_barrier * sizeof(int));
        s->S.barrier = d;
    } else {
        s->S.barrier = nullptr;
    }
    s->S.nb = n_barrier;
    s->S.n_layers = n_layers;
    s->drop_graphs();
    return upload_nav(s);
}

int fp_set_state(fp_sim *s, const float *h, const float *hu, const float *hv) {
    if (!s) return FP_EINVAL;
    if (!h || !hu || !hv) return s->fail(FP_EINVAL, "null state array");
    const int p = s->par;
    cudaError_t e;
    if ((e = put_plane(s, s->S.h[p], h)) != cudaSuccess) return s->cuda_fail(e, "h upload");
    if ((e = put_plane(s, s->S.hu[p], hu)) != cudaSuccess) return s->cuda_fail(e, "hu upload");
    if ((e = put_plane(s, s->S.hv[p], hv)) != cudaSuccess) return s->cuda_fail(e, "hv upload");
    cudaMemsetAsync(s->S.bflux, 0, (2 * (size_t)s->S.nx + 2 * (size_t)s->S.ny) * sizeof(double), s->stream);
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return s->cuda_fail(e, "state upload");
    s->need_prepare = true;
    return FP_OK;
}

int fp_set_time(fp_sim *s, int64_t t_ticks, int64_t step) {
    if (!s) return FP_EINVAL;
    if (t_ticks < 0 || step < 0) return s->fail(FP_EINVAL, "negative time or step");
    s->pending_time = true;
    s->pend_t = t_ticks;
    s->pend_step = step;
    s->need_prepare = true;
    return FP_OK;
}

int fp_set_barrier_progress(fp_sim *s, int64_t total_bags, int64_t applied_layers) {
    if (!s) return FP_EINVAL;
    if (total_bags < 0 || applied_layers < 0) return s->fail(FP_EINVAL, "negative barrier progress");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "sync");
    FpCounters c;
    s->copy(&c, s->S.cnt, sizeof(c));
    c.total_bags = (unsigned long long)total_bags;
    c.bags_snap = (unsigned long long)total_bags;
    c.applied = (unsigned long long)applied_layers;
    e = s->copy(s->S.cnt, &c, sizeof(c));
    if (e != cudaSuccess) return s->cuda_fail(e, "barrier progress");
    return FP_OK;
}

int fp_add_pedestrians(fp_sim *s, const fp_ped *peds, int32_t count) {
    if (!s) return FP_EINVAL;
    if (count < 0 || (count > 0 && !peds)) return s->fail(FP_EINVAL, "bad pedestrian arguments");
    if (count == 0) return FP_OK;
    cudaError_t e = drop_hash(s);
    if (e != cudaSuccess) return s->cuda_fail(e, "hash reset");
    // the record count of B and the ids issued (doors admit visitors on the
    // device): known on the host since a clear or an add, else read
    int nb0 = s->nb_known, ids0 = s->ids_known;
    if (nb0 < 0 || ids0 < 0) {
        FpCounters c;
        if ((e = s->copy(&c, s->S.cnt, sizeof(c))) != cudaSuccess) return s->cuda_fail(e, "counters read");
        nb0 = c.nB;
        ids0 = c.n_ids;
    }
    if ((long long)ids0 + count > s->S.cap || (long long)nb0 + count > s->S.cap)
        return s->fail(FP_EOVERFLOW, "pedestrian capacity exceeded");
    // upload, ids and the new record count (set by the kernel), then one read
    // back for the walkability check (which also waits for the upload)
    e = cudaMemcpyAsync(s->S.pedB + 2 * (size_t)nb0, peds, (size_t)count * sizeof(fp_ped), cudaMemcpyDefault,
                        s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "pedestrian upload");
    fp_launch_assign_ids(s->S, nb0, ids0, count, s->stream);
    int bad = 0;
    if ((e = s->copy(&bad, &s->S.cnt->bad_ped, sizeof(int))) != cudaSuccess) return s->cuda_fail(e, "assign ids");
    if (bad) {
        int zero = 0;
        s->copy(&s->S.cnt->bad_ped, &zero, sizeof(int));
        s->copy(&s->S.cnt->nB, &nb0, sizeof(int));  // the records stay out
        s->copy(&s->S.cnt->n_ids, &ids0, sizeof(int));
        s->nb_known = nb0;
        s->ids_known = ids0;
        return s->fail(FP_EINVAL, "a pedestrian stands outside the domain or in a non-walkable cell");
    }
    s->nb_known = nb0 + count;
    s->ids_known = ids0 + count;
    return FP_OK;
}

int fp_clear_pedestrians(fp_sim *s) {
    if (!s) return FP_EINVAL;
    cudaError_t e = drop_hash(s);
    if (e == cudaSuccess) {
        fp_launch_clear_peds(s->S, s->stream);  // stream-ordered: no host round trip
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return s->cuda_fail(e, "clear");
    s->nb_known = 0;
    s->ids_known = 0;
    return FP_OK;
}

int fp_step(fp_sim *s, int32_t n_steps) {
    if (!s) return FP_EINVAL;
    if (n_steps < 0) return s->fail(FP_EINVAL, "negative step count");
    if (n_steps > 0) s->nb_known = s->ids_known = -1;  // exits and door admissions change them
    if (s->need_prepare) {
        int rc = prepare(s);
        if (rc != FP_OK) return rc;
    }
    if (s->profiling) return step_profiled(s, n_steps);
    if (s->mode == FP_MODE_PERSISTENT) {
        const cudaError_t eh = drop_hash(s);  // the persistent kernel hashes B itself
        if (eh != cudaSuccess) return s->cuda_fail(eh, "hash reset");
        int left = n_steps;
        while (left > 0) {
            const int n = left < kPersistSteps ? left : kPersistSteps;
            cudaError_t e = fp_launch_persistent(s->S, s->par, s->slot, n, s->grid_bar, s->persist_ctas, s->stream);
            if (e != cudaSuccess) return s->cuda_fail(e, "persistent launch");
            if (n & 1) s->par ^= 1;
            s->slot = (s->slot + n) & 3;
            left -= n;
        }
        return FP_OK;
    }
    int left = n_steps;
    while (left > 0) {
        if (left >= kGraphSteps) {
            cudaGraphExec_t &g = s->graphs[s->hashed ? 1 : 0][s->slot];
            if (!g) {
                cudaGraph_t graph;
                cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) return s->cuda_fail(e, "begin capture");
                int p = s->par, sl = s->slot;
                for (int k = 0; k < kGraphSteps; ++k) {
                    launch_step(s, p, sl);
                    p ^= 1;
                    sl = (sl + 1) & 3;
                }
                e = cudaStreamEndCapture(s->stream, &graph);
                if (e != cudaSuccess) return s->cuda_fail(e, "end capture");
                e = cudaGraphInstantiate(&g, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) { g = nullptr; return s->cuda_fail(e, "graph instantiate"); }
            }
            cudaError_t e = cudaGraphLaunch(g, s->stream);
            if (e != cudaSuccess) return s->cuda_fail(e, "graph launch");
            s->hashed = s->hash_ahead;  // its last step hashed the records for the next
            left -= kGraphSteps;  // 64 steps: parity and slot return to their start values
        } else {
            launch_step(s, s->par, s->slot);
            s->par ^= 1;
            s->slot = (s->slot + 1) & 3;
            left -= 1;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return s->cuda_fail(e, "step launch");
    return FP_OK;
}

int fp_set_tuning(fp_sim *s, int32_t tile_rows, int32_t ped_lanes) {
    if (!s) return FP_EINVAL;
    if ((tile_rows != 8 && tile_rows != 16 && tile_rows != 32) ||
        (ped_lanes != 1 && ped_lanes != 2 && ped_lanes != 4 && ped_lanes != 8 && ped_lanes != 16))
        return s->fail(FP_EINVAL, "tile_rows must be 8, 16 or 32 and ped_lanes 1, 2, 4, 8 or 16");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "tuning switch");
    s->tile_rows = tile_rows;
    s->ped_lanes = ped_lanes;
    s->drop_graphs();
    return FP_OK;
}

int fp_set_hash_ahead(fp_sim *s, int32_t on) {
    if (!s) return FP_EINVAL;
    if (on != 0 && on != 1) return s->fail(FP_EINVAL, "hash-ahead is 0 or 1");
    if ((on != 0) == s->hash_ahead) return FP_OK;
    cudaError_t e = drop_hash(s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "hash-ahead switch");
    s->hash_ahead = on != 0;
    s->drop_graphs();  // the graphs' steps hash ahead or not
    return FP_OK;
}

int fp_set_step_mode(fp_sim *s, int32_t mode) {
    if (!s) return FP_EINVAL;
    if (mode != FP_MODE_KERNELS && mode != FP_MODE_PERSISTENT) return s->fail(FP_EINVAL, "unknown step mode");
    if (mode == FP_MODE_PERSISTENT && s->persist_ctas <= 0)
        return s->fail(FP_EINVAL, "cooperative launch unavailable on this device");
    if (mode == FP_MODE_PERSISTENT && s->S.order == 2)
        return s->fail(FP_EINVAL, "the second-order update runs in FP_MODE_KERNELS only");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "mode switch");
    s->mode = mode;
    return FP_OK;
}

int fp_set_fixed_dt(fp_sim *s, double dt_seconds) {
    if (!s) return FP_EINVAL;
    if (!(dt_seconds >= 0.0) || dt_seconds > 1.0) return s->fail(FP_EINVAL, "fixed dt must lie in [0, 1] s");
    long long ticks = llround(dt_seconds * 1048576.0);
    if (dt_seconds > 0.0 && ticks < 1) ticks = 1;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "fixed dt switch");
    s->S.dt_fixed = ticks;
    s->drop_graphs();
    return FP_OK;
}

int fp_surrogate_advance(fp_sim *s, fp_surrogate *sur, int32_t n_windows, const fp_surrogate_guard *guard,
                         fp_surrogate_stats *st) {
    if (!s) return FP_EINVAL;
    if (!sur || !guard || !st || n_windows < 0) return s->fail(FP_EINVAL, "null surrogate, guard or stats");
    if (s->S.dt_fixed <= 0) return s->fail(FP_EINVAL, "the surrogate window needs a fixed time step (fp_set_fixed_dt)");
    if (s->S.has_discharge) return s->fail(FP_EINVAL, "the surrogate window does not take a discharge breach");
    if (s->S.order == 2) return s->fail(FP_EINVAL, "the surrogate window stands in for the first-order update");
    if (!(guard->mass_tol >= 0.0f) || !(guard->check_tol >= 0.0f) || !(guard->fix_tol >= 0.0f) ||
        guard->check_every < 0 ||
        guard->suspend_windows < 0)
        return s->fail(FP_EINVAL, "invalid guard parameters");
    if (s->need_prepare) {
        const int rc = prepare(s);
        if (rc != FP_OK) return rc;
    }
    s->nb_known = -1;
    int rc = ensure_window(s);
    if (rc != FP_OK) return rc;
    {
        const cudaError_t eh = drop_hash(s);  // the window's steps hash B themselves
        if (eh != cudaSuccess) return s->cuda_fail(eh, "hash reset");
    }
    fp_sim::Window &W = s->win;
    const FpSim &S = s->S;
    const int nt = W.tiles_x * W.tiles_y;
    const int kIn = FP_SUR_TILE + 2 * FP_SUR_HALO;
    const size_t pbytes = s->plane_elems() * sizeof(float);
    const int ftx = (S.nx + FP_TX - 1) / FP_TX, fty = (S.ny + s->tile_rows - 1) / s->tile_rows;
    std::vector<unsigned char> flag(nt), fail(nt), mask(W.ftiles), keep(nt);
    std::vector<int> list(nt);
    std::vector<float> resid(nt);
    cudaError_t e = cudaSuccess;
    for (int w = 0; w < n_windows; ++w) {
        const int par = s->par, slot = s->slot;
        FpClock c0;
        e = s->copy(&c0, &S.clock[slot], sizeof(c0));
        if (e != cudaSuccess) return s->cuda_fail(e, "window clock");
        if (c0.t + (long long)FP_SUR_WINDOW * S.dt_fixed > S.t_end) break;
        const bool check = guard->check_every > 0 && (W.done + 1) % guard->check_every == 0;
        const bool plain = W.suspend > 0;
        float *state[3] = {S.h[par], S.hu[par], S.hv[par]};
        float *other[3] = {S.h[par ^ 1], S.hu[par ^ 1], S.hv[par ^ 1]};
        for (int k = 0; k < 3; ++k) cudaMemcpyAsync(W.u0[k], state[k], pbytes, cudaMemcpyDeviceToDevice, s->stream);
        cudaMemsetAsync(W.clock, 0, 4 * sizeof(FpClock), s->stream);
        cudaMemcpyAsync(&W.clock[slot], &S.clock[slot], sizeof(FpClock), cudaMemcpyDeviceToDevice, s->stream);
        // 1-2. dry tiles and the net's tiles
        int count = 0;
        if (!plain) {
            fp_launch_sur_classify(S, par, &W.clock[slot], W.tiles_x, W.tiles_y, W.wet, s->stream);
            fp_launch_sur_compact(W.wet, nt, W.list, W.batch_of, W.count, s->stream);
            e = s->copy(&count, W.count, sizeof(int));
            if (e != cudaSuccess) return s->cuda_fail(e, "window tile count");
            if (count > 0) {
                // the net on its own stream, beside the pedestrian steps: both
                // read only the start state (the input packing reads z before
                // the steps may raise it)
                cudaEventRecord(W.ev_start, s->stream);
                cudaStreamWaitEvent(W.net_stream, W.ev_start, 0);
                fp_launch_sur_input(S, W.u0[0], W.u0[1], W.u0[2], W.list, count, W.tiles_x, W.x16, W.net_stream);
                cudaEventRecord(W.ev_input, W.net_stream);
                e = fp_sur_forward_packed(sur, W.x16, count, kIn, kIn, W.dU, W.net_stream);
                if (e != cudaSuccess) return s->cuda_fail(e, "surrogate forward");
                cudaEventRecord(W.ev_net, W.net_stream);
                cudaStreamWaitEvent(s->stream, W.ev_input, 0);
            }
        }
        // 3. pedestrians over the window on the start state
        for (int k = 0; k < 3; ++k) cudaMemcpyAsync(other[k], W.u0[k], pbytes, cudaMemcpyDeviceToDevice, s->stream);
        for (int k = 0; k < FP_SUR_WINDOW; ++k) {
            launch_window_step(s, s->par, s->slot);
            s->par ^= 1;
            s->slot = (s->slot + 1) & 3;
        }
        // 4. apply the net's change, guard
        std::fill(flag.begin(), flag.end(), (unsigned char)(plain || check ? 1 : 0));
        std::fill(keep.begin(), keep.end(), (unsigned char)0);  // net tiles the guard accepted
        if (count > 0) {
            cudaStreamWaitEvent(s->stream, W.ev_net, 0);
            cudaMemsetAsync(W.count + 1, 0, sizeof(int), s->stream);
            fp_launch_sur_apply(S, par, W.u0[0], W.u0[1], W.u0[2], W.dU, W.list, W.batch_of, count, W.tiles_x,
                                &W.clock[slot], guard->mass_tol, guard->fix_tol, W.fail, W.resid, W.count + 1,
                                s->stream);
            e = s->copy(fail.data(), W.fail, count);
            if (e == cudaSuccess) e = s->copy(resid.data(), W.resid, count * sizeof(float));
            if (e == cudaSuccess) e = s->copy(list.data(), W.list, count * sizeof(int));
            if (e != cudaSuccess) return s->cuda_fail(e, "window guard");
            for (int b = 0; b < count; ++b) {
                st->max_residual = std::max(st->max_residual, (double)resid[b]);
                keep[list[b]] = fail[b] ? 0 : 1;
                if (fail[b]) {
                    flag[list[b]] = 1;
                    st->tiles_fallback += 1;
                    st->fail_mass += fail[b] & 1;
                    st->fail_courant += (fail[b] >> 1) & 1;
                    st->fail_nonfinite += (fail[b] >> 2) & 1;
                }
            }
        }
        st->windows += 1;
        st->tiles += nt;
        st->tiles_net += count;
        if (plain || check) st->tiles_plain += nt;
        // 5-6. plain update of the flagged tiles (grown by the window) from the start state
        bool any = false;
        for (unsigned char f : flag) any |= f != 0;
        if (any) {
            const unsigned char *dmask = nullptr;
            if (!(plain || check)) {
                std::fill(mask.begin(), mask.end(), (unsigned char)0);
                for (int t = 0; t < nt; ++t) {
                    if (!flag[t]) continue;
                    const int xa = std::max(0, (t % W.tiles_x) * FP_SUR_TILE - FP_SUR_WINDOW);
                    const int xb = std::min(S.nx, (t % W.tiles_x + 1) * FP_SUR_TILE + FP_SUR_WINDOW);
                    const int ya = std::max(0, (t / W.tiles_x) * FP_SUR_TILE - FP_SUR_WINDOW);
                    const int yb = std::min(S.ny, (t / W.tiles_x + 1) * FP_SUR_TILE + FP_SUR_WINDOW);
                    for (int fy = ya / s->tile_rows; fy <= (yb - 1) / s->tile_rows && fy < fty; ++fy)
                        for (int fx = xa / FP_TX; fx <= (xb - 1) / FP_TX && fx < ftx; ++fx) mask[fy * ftx + fx] = 1;
                }
                e = s->copy(W.mask, mask.data(), W.ftiles);
                if (e != cudaSuccess) return s->cuda_fail(e, "fallback mask");
                dmask = W.mask;
            }
            for (int p = 0; p < 2; ++p)
                for (int k = 0; k < 3; ++k)
                    cudaMemcpyAsync(W.fb[p][k], W.u0[k], pbytes, cudaMemcpyDeviceToDevice, s->stream);
            FpSim F = S;
            for (int p = 0; p < 2; ++p) {
                F.h[p] = W.fb[p][0];
                F.hu[p] = W.fb[p][1];
                F.hv[p] = W.fb[p][2];
                F.occ[p] = W.fb_occ;
                F.blk_wet[p] = nullptr;  // the fallback planes start from the window's start state
            }
            F.clock = W.clock;
            F.bflux = W.bflux;
            F.tile_mask = dmask;
            int p = par, sl = slot;
            for (int k = 0; k < FP_SUR_WINDOW; ++k) {
                cudaMemsetAsync(W.fb_occ, 0, s->plane_elems() * sizeof(unsigned short), s->stream);
                if (S.coupling) fp_launch_sur_occupancy(F, W.fb_occ, s->stream);
                fp_launch_flood(F, p, sl, s->tile_rows, s->stream);
                p ^= 1;
                sl = (sl + 1) & 3;
            }
            if (check) {
                // the error of what the surrogate path keeps: net tiles the guard
                // accepted (rejected ones are replaced by the plain result)
                unsigned bits = 0;
                e = s->copy(W.keep, keep.data(), nt);
                if (e != cudaSuccess) return s->cuda_fail(e, "check tiles");
                cudaMemsetAsync(W.maxdiff, 0, sizeof(unsigned), s->stream);
                fp_launch_sur_diff(S, S.h[par], W.fb[par][0], W.keep, W.tiles_x, W.maxdiff, s->stream);
                e = s->copy(&bits, W.maxdiff, sizeof(unsigned));
                if (e != cudaSuccess) return s->cuda_fail(e, "plain check");
                float err;
                memcpy(&err, &bits, sizeof(err));
                st->checks += 1;
                st->max_check_error = std::max(st->max_check_error, (double)err);
                if (!(err <= guard->check_tol)) {
                    st->checks_failed += 1;
                    W.suspend = guard->suspend_windows + 1;  // this window's decrement below
                }
            }
            e = s->copy(W.flag, flag.data(), nt);
            if (e != cudaSuccess) return s->cuda_fail(e, "fallback flags");
            fp_launch_sur_merge(S, par, W.fb[par][0], W.fb[par][1], W.fb[par][2], W.flag, W.tiles_x, W.tiles_y,
                                s->stream);
        }
        // the clock of the window's end takes the wave speed and wet flag of
        // the new water state (the window's own steps carried the start's)
        cudaMemsetAsync(&S.clock[s->slot].smax_bits, 0, sizeof(unsigned), s->stream);
        fp_launch_init_clock(S, s->par, s->slot, s->stream);
        if (W.suspend > 0) W.suspend -= 1;
        W.done += 1;
    }
    e = s->reset_water_flags();  // the window wrote the water state
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return s->cuda_fail(e, "surrogate window");
    if (fp_sur_error_bits(sur) & FP_ERR_TIMEOUT) return s->fail(FP_ETIMEOUT, "tensor-core completion wait timed out");
    return fp_synchronize(s);
}

int fp_set_profiling(fp_sim *s, int32_t on) {
    if (!s) return FP_EINVAL;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "profiling switch");
    s->profiling = on != 0;
    for (double &v : s->prof) v = 0.0;
    if (s->profiling) {
        const size_t nb = s->flag_blocks();
        if (!s->blk_runs && !(s->blk_runs = s->dalloc<unsigned>(nb))) return s->fail(FP_ENOMEM, "profile counters");
        e = cudaMemsetAsync(s->blk_runs, 0, nb * sizeof(unsigned), s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return s->cuda_fail(e, "profile counters");
    }
    s->S.blk_runs = s->profiling ? s->blk_runs : nullptr;
    return FP_OK;
}

// After a device error: the error word and the transient per-step structures
// (bin counts, evacuee counts, the hash made ahead) back to their between-step
// values, so that the handle takes new state and steps again.
static cudaError_t clear_device_error(fp_sim *s) {
    const FpSim &S = s->S;
    s->hashed = false;
    cudaError_t e = cudaMemsetAsync(S.bin_count, 0, ((size_t)S.nbins + 1) * sizeof(int), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.tile_sum, 0, (size_t)fp_scan_tiles(S.nbins) * sizeof(int), s->stream);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p)
        e = cudaMemsetAsync(S.occ[p], 0, s->plane_elems() * sizeof(unsigned short), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&S.cnt->err, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&S.cnt->flood_ticket, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    s->need_prepare = true;
    return e;
}

int fp_synchronize(fp_sim *s) {
    if (!s) return FP_EINVAL;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "synchronize");
    unsigned err = 0;
    e = s->copy(&err, &s->S.cnt->err, sizeof(err));
    if (e != cudaSuccess) return s->cuda_fail(e, "error word");
    if (err == 0) return FP_OK;
    e = clear_device_error(s);
    if (e != cudaSuccess) return s->cuda_fail(e, "error reset");
    if (err & FP_ERR_TIMEOUT) return s->fail(FP_ETIMEOUT, "a bounded device wait timed out");
    if (err & FP_ERR_OCC_OVERFLOW) return s->fail(FP_EOVERFLOW, "more than 65535 evacuees in one cell");
    if (err & FP_ERR_NAN) return s->fail(FP_ENAN, "non-finite water state");
    if (err & FP_ERR_CAPACITY) return s->fail(FP_EOVERFLOW, "a door admission exceeded the pedestrian capacity");
    return s->fail(FP_ECUDA, "device error bits set");
}

int fp_set_barrier_wait_limit(fp_sim *s, int32_t polls) {
    if (!s) return FP_EINVAL;
    if (polls < 0) return s->fail(FP_EINVAL, "negative poll limit");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "wait limit switch");
    s->S.barrier_polls = polls;
    s->drop_graphs();
    return FP_OK;
}

int fp_read_state(fp_sim *s, int32_t which, void *dst, size_t bytes) {
    if (!s) return FP_EINVAL;
    if (!dst) return s->fail(FP_EINVAL, "null destination");
    if (s->need_prepare) {
        int rc = prepare(s);
        if (rc != FP_OK) return rc;
    }
    const FpSim &S = s->S;
    const size_t n = (size_t)S.nx * S.ny;
    cudaError_t e = cudaSuccess;
    switch (which) {
        case FP_FIELD_H:
        case FP_FIELD_HU:
        case FP_FIELD_HV:
        case FP_FIELD_Z: {
            if (bytes < n * 4) return s->fail(FP_EINVAL, "destination too small");
            const float *src = which == FP_FIELD_H ? S.h[s->par] : which == FP_FIELD_HU ? S.hu[s->par]
                               : which == FP_FIELD_HV ? S.hv[s->par] : S.z;
            e = get_plane(s, dst, src);
            break;
        }
        case FP_FIELD_PEDS: {
            int n_ids = 0;
            if ((e = s->copy(&n_ids, &S.cnt->n_ids, sizeof(int))) != cudaSuccess) break;
            if (bytes < (size_t)n_ids * sizeof(fp_ped)) return s->fail(FP_EINVAL, "destination too small");
            fp_launch_read_peds(S, s->read_buf, n_ids, s->stream);
            if (n_ids)
                e = cudaMemcpyAsync(dst, s->read_buf, (size_t)n_ids * sizeof(fp_ped), cudaMemcpyDefault, s->stream);
            break;
        }
        case FP_FIELD_COUNTERS: {
            if (bytes < sizeof(fp_counters)) return s->fail(FP_EINVAL, "destination too small");
            FpCounters c;
            FpClock k;
            cudaStreamSynchronize(s->stream);
            s->copy(&c, S.cnt, sizeof(c));
            e = s->copy(&k, &S.clock[s->slot], sizeof(k));
            fp_counters o;
            memset(&o, 0, sizeof(o));
            o.t_ticks = k.t;
            o.step = k.step;
            o.n_exited = (int64_t)c.n_exited;
            o.n_active = (int64_t)c.n_ids - (int64_t)c.n_exited - (int64_t)c.n_left;
            o.n_ids = c.n_ids;
            o.n_entered = (int64_t)c.n_entered;
            o.n_left = (int64_t)c.n_left;
            o.total_bags = (int64_t)c.total_bags;
            o.applied_layers = (int64_t)c.applied;
            o.neg_depth = (int64_t)c.neg_depth;
            for (int q = 0; q < 5; ++q) o.hist[q] = (int64_t)c.hist[q];
            o.wet = k.wet;
            o.error_flags = c.err;
            o.ped_updates = (int64_t)c.ped_updates;
            o.cfl_exceeded = (int64_t)c.cfl_over;
            if (e == cudaSuccess) e = s->copy(dst, &o, sizeof(o));
            break;
        }
        case FP_FIELD_NAV: {
            if (bytes < 3 * n) return s->fail(FP_EINVAL, "destination too small");
            for (int g = 0; g < 3 && e == cudaSuccess; ++g)
                e = cudaMemcpyAsync(static_cast<uint8_t *>(dst) + g * n, S.nav[g], n, cudaMemcpyDefault, s->stream);
            break;
        }
        case FP_FIELD_MASS: {
            if (bytes < 2 * sizeof(double)) return s->fail(FP_EINVAL, "destination too small");
            fp_launch_mass(S, s->par, s->stream);
            double tmp[2];
            e = cudaMemcpyAsync(tmp, &S.cnt->mass, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
            if (e == cudaSuccess) e = s->copy(dst, tmp, sizeof(tmp));
            break;
        }
        case FP_FIELD_HR_MAX: {
            if (bytes < sizeof(float)) return s->fail(FP_EINVAL, "destination too small");
            fp_launch_hr_max(S, s->par, s->stream);
            unsigned bits = 0;
            e = cudaMemcpyAsync(&bits, &S.cnt->hr_max_bits, sizeof(bits), cudaMemcpyDeviceToHost, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
            if (e == cudaSuccess) e = s->copy(dst, &bits, sizeof(float));
            break;
        }
        case FP_FIELD_PROFILE: {
            if (bytes < sizeof(s->prof)) return s->fail(FP_EINVAL, "destination too small");
            e = s->copy(dst, s->prof, sizeof(s->prof));
            break;
        }
        default:
            return s->fail(FP_EINVAL, "unknown field");
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "read_state");
    return FP_OK;
}

}  // extern "C"

struct fp_batch {
    std::vector<fp_sim *> sims;
    int n = 0, total_runs = 0, total_rec = 0, max_scan_tiles = 0;
    FpSim *d_sims = nullptr;
    // flood runs of the persistent kernel (64 x kBatchPersistRows) and record slots of each member
    int *d_run_off = nullptr, *d_rec_off = nullptr;
    // per-step kernels: members grouped by their launch shapes when the batch
    // was made (flood run height, lanes per pedestrian), device lists
    FpBatchGroups fg{}, pg{};
    std::vector<FpSim> h_sims;
    cudaStream_t stream = nullptr, stream2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t graphs[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<void *> allocs;
    int mode = FP_MODE_KERNELS;
    int ctas = 0;            // CTAs of the persistent launch
    unsigned *bar = nullptr;  // grid barrier word + pedestrian and flood tickets (8 words)
};

static void batch_launch_step(fp_batch *b, int par, int slot) {
    fp_launch_batch_peds(b->d_sims, b->d_rec_off, b->n, b->total_rec, b->max_scan_tiles, b->pg, par, slot,
                         b->stream, b->stream2, b->ev_fork, true);
    cudaStreamWaitEvent(b->stream2, b->ev_fork, 0);
    fp_launch_flood_batch(b->d_sims, b->fg, par, slot, b->stream);
    fp_launch_batch_peds(b->d_sims, b->d_rec_off, b->n, b->total_rec, b->max_scan_tiles, b->pg, par, slot,
                         b->stream, b->stream2, b->ev_fork, false);
    cudaEventRecord(b->ev_join, b->stream2);
    cudaStreamWaitEvent(b->stream, b->ev_join, 0);
}

extern "C" {

int fp_batch_create(fp_sim *const *sims, int32_t n, fp_batch **out) {
    if (!sims || !out || n < 1) {
        g_create_error = "fp_batch_create: need n >= 1 simulations";
        return FP_EINVAL;
    }
    *out = nullptr;
    fp_batch *b = new fp_batch();
    b->n = n;
    std::vector<int> run_off(n + 1, 0), rec_off(n + 1, 0);
    for (int k = 0; k < n; ++k) {
        fp_sim *m = sims[k];
        if (!m) { delete b; g_create_error = "fp_batch_create: null member"; return FP_EINVAL; }
        if (m->S.order == 2) {
            delete b;
            g_create_error = "fp_batch_create: a member uses the second-order update (per-step kernels only)";
            return FP_EINVAL;
        }
        b->sims.push_back(m);
        const int runs = ((m->S.nx + FP_TX - 1) / FP_TX) * ((m->S.ny + kBatchPersistRows - 1) / kBatchPersistRows);
        run_off[k + 1] = run_off[k] + runs;
        const int cap = std::max(1, m->S.cap);
        rec_off[k + 1] = rec_off[k] + ((cap + 255) / 256) * 256;
        b->max_scan_tiles = std::max(b->max_scan_tiles, fp_scan_tiles(m->S.nbins));
    }
    b->total_runs = run_off[n];
    b->total_rec = rec_off[n];
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        b->allocs.push_back(p);
        return p;
    };
    b->d_sims = static_cast<FpSim *>(alloc(sizeof(FpSim) * n));
    b->d_run_off = static_cast<int *>(alloc(sizeof(int) * (n + 1)));
    b->d_rec_off = static_cast<int *>(alloc(sizeof(int) * (n + 1)));
    b->bar = static_cast<unsigned *>(alloc(8 * sizeof(unsigned)));
    if (!b->d_sims || !b->d_run_off || !b->d_rec_off || !b->bar) {
        fp_batch_destroy(b);
        g_create_error = "fp_batch_create: device allocation failed";
        return FP_ENOMEM;
    }
    cudaMemcpy(b->d_run_off, run_off.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_rec_off, rec_off.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
    // shape groups: member lists and work-item offsets per flood run height
    // and per lane count (each member's fp_set_tuning shape)
    auto build_groups = [&](FpBatchGroups &G, const int *values, int nvals, bool flood) -> bool {
        for (int g = 0; g < nvals; ++g) {
            std::vector<int> mem, off(1, 0);
            for (int k = 0; k < n; ++k) {
                const fp_sim *m = b->sims[k];
                if ((flood ? m->tile_rows : m->ped_lanes) != values[g]) continue;
                mem.push_back(k);
                const int items = flood ? ((m->S.nx + FP_TX - 1) / FP_TX) * ((m->S.ny + values[g] - 1) / values[g])
                                        : (rec_off[k + 1] - rec_off[k]) * values[g] / 256;
                off.push_back(off.back() + items);
            }
            G.n[g] = (int)mem.size();
            G.total[g] = off.back();
            if (mem.empty()) continue;
            int *dm = static_cast<int *>(alloc(sizeof(int) * mem.size()));
            int *dof = static_cast<int *>(alloc(sizeof(int) * off.size()));
            if (!dm || !dof) return false;
            cudaMemcpy(dm, mem.data(), sizeof(int) * mem.size(), cudaMemcpyHostToDevice);
            cudaMemcpy(dof, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice);
            G.members[g] = dm;
            G.off[g] = dof;
        }
        return true;
    };
    if (!build_groups(b->fg, kBatchFloodRows, 3, true) || !build_groups(b->pg, kBatchPedLanes, 5, false)) {
        fp_batch_destroy(b);
        g_create_error = "fp_batch_create: device allocation failed";
        return FP_ENOMEM;
    }
    b->h_sims.resize(n);
    cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&b->stream2, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        fp_batch_destroy(b);
        g_create_error = "fp_batch_create: CUDA error";
        return FP_ECUDA;
    }
    *out = b;
    return FP_OK;
}

int fp_batch_step(fp_batch *b, int32_t n_steps) {
    if (!b || n_steps < 0) return FP_EINVAL;
    const int par = b->sims[0]->par, slot = b->sims[0]->slot;
    for (int k = 0; k < b->n; ++k) {
        fp_sim *m = b->sims[k];
        m->nb_known = -1;
        cudaError_t e = drop_hash(m);  // the batch kernels hash B themselves
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) return m->cuda_fail(e, "batch member sync");
        if (m->need_prepare) {
            int rc = prepare(m);
            if (rc != FP_OK) return rc;
        }
        if (m->par != par || m->slot != slot) {
            g_create_error = "fp_batch_step: members are at different step parities";
            return FP_EINVAL;
        }
        b->h_sims[k] = m->S;
        b->h_sims[k].blk_runs = nullptr;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_sims, b->h_sims.data(), sizeof(FpSim) * b->n, cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host vectors may change at the next call
    if (e != cudaSuccess) {
        g_create_error = "fp_batch_step: descriptor upload failed";
        return FP_ECUDA;
    }
    int p = par, sl = slot, left = n_steps;
    while (left > 0 && b->mode == FP_MODE_PERSISTENT) {
        const int k = std::min(left, kPersistSteps);
        e = fp_launch_batch_persistent(b->d_sims, b->d_run_off, b->d_rec_off, b->n, b->total_runs, b->total_rec,
                                       b->max_scan_tiles, p, sl, k, b->bar, b->ctas, b->stream);
        if (e != cudaSuccess) break;
        p ^= k & 1;
        sl = (sl + k) & 3;
        left -= k;
    }
    while (left > 0) {
        if (left >= kGraphSteps) {
            cudaGraphExec_t &g = b->graphs[sl];
            if (!g) {
                cudaGraph_t graph;
                e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) break;
                int pp = p, ss = sl;
                for (int k = 0; k < kGraphSteps; ++k) {
                    batch_launch_step(b, pp, ss);
                    pp ^= 1;
                    ss = (ss + 1) & 3;
                }
                e = cudaStreamEndCapture(b->stream, &graph);
                if (e != cudaSuccess) break;
                e = cudaGraphInstantiate(&g, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) { g = nullptr; break; }
            }
            e = cudaGraphLaunch(g, b->stream);
            if (e != cudaSuccess) break;
            left -= kGraphSteps;
        } else {
            batch_launch_step(b, p, sl);
            p ^= 1;
            sl = (sl + 1) & 3;
            left -= 1;
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_create_error = std::string("fp_batch_step: ") + cudaGetErrorString(e);
        return FP_ECUDA;
    }
    for (fp_sim *m : b->sims) {
        m->par = p;
        m->slot = sl;
    }
    return FP_OK;
}

int fp_batch_set_step_mode(fp_batch *b, int32_t mode) {
    if (!b) return FP_EINVAL;
    if (mode != FP_MODE_KERNELS && mode != FP_MODE_PERSISTENT) {
        g_create_error = "fp_batch_set_step_mode: unknown step mode";
        return FP_EINVAL;
    }
    if (mode == FP_MODE_PERSISTENT) {
        if (b->ctas <= 0) b->ctas = fp_batch_persistent_ctas();
        if (b->ctas <= 0) {
            g_create_error = "fp_batch_set_step_mode: cooperative launch unavailable on this device";
            return FP_EINVAL;
        }
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("fp_batch_set_step_mode: ") + cudaGetErrorString(e);
        return FP_ECUDA;
    }
    b->mode = mode;
    return FP_OK;
}

int fp_batch_synchronize(fp_batch *b) {
    if (!b) return FP_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("fp_batch_synchronize: ") + cudaGetErrorString(e);
        return FP_ECUDA;
    }
    // every member's error is read (each is reported once); after any error the
    // hashing state of every member is reset: a persistent launch that gave up
    // leaves all members part-way through a step
    int first = FP_OK;
    for (fp_sim *m : b->sims) {
        const int rc = fp_synchronize(m);
        if (rc != FP_OK && first == FP_OK) {
            first = rc;
            g_create_error = m->err;
        }
    }
    if (first != FP_OK) {
        for (fp_sim *m : b->sims) {
            e = clear_device_error(m);
            if (e != cudaSuccess) {
                g_create_error = std::string("fp_batch_synchronize: ") + cudaGetErrorString(e);
                return FP_ECUDA;
            }
        }
    }
    return first;
}

int fp_batch_destroy(fp_batch *b) {
    if (!b) return FP_EINVAL;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &g : b->graphs)
        if (g) cudaGraphExecDestroy(g);
    for (void *p : b->allocs) cudaFree(p);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->stream2) cudaStreamDestroy(b->stream2);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
    return FP_OK;
}

int fp_destroy(fp_sim *s) {
    if (!s) return FP_EINVAL;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->stream2) cudaStreamSynchronize(s->stream2);
    if (s->win.net_stream) cudaStreamSynchronize(s->win.net_stream);
    s->drop_graphs();
    for (void *p : s->allocs) cudaFree(p);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    if (s->stream2) cudaStreamDestroy(s->stream2);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
    if (s->win.net_stream) cudaStreamDestroy(s->win.net_stream);
    for (cudaEvent_t e : {s->win.ev_start, s->win.ev_input, s->win.ev_net})
        if (e) cudaEventDestroy(e);
    delete s;
    return FP_OK;
}

const char *fp_last_error(const fp_sim *s) { return s ? s->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

void fp_note_error(const char *msg) { g_create_error = msg; }

extern "C" {

}  // extern "C"
