// cm_api.cu -- C ABI and host runtime of libcm (declared in include/cm.h).
//
// The runtime owns a context's scratch (the second ping-pong image, energy
// partials, a pinned readback slot) and a cached CUDA graph per solve
// configuration.  The graph holds the whole outer loop of Alg. 3: the initial
// energy, then a conditional WHILE node whose body is one full cycle (every
// phase of every level, the FP64 energy) followed by the stopping test of
// Eq. (reerr) on the device, which sets the loop condition.  The host reads
// the solve's state back once, after the loop.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <string>

#include <vector>

#include "../../include/cm.h"
#include "cm_batched.h"
#include "cm_cnn.h"
#include "cm_kernels.h"
#include "cm_fft.h"
#include "cm_recon.h"

struct GraphKey {
    const float* S;
    const float* R;
    const float* f;
    int H, W, kind, levels, ncolors, G, K, use_paper, one_step, vcycle, coarse_spec, coarse_dmax,
        block_sides, coarse_ncolors, shapes;
    float alpha;
    double tol;
    int cycles, trace_cap;
    bool operator==(const GraphKey& o) const { return memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

// Tracing: an NVTX range (header-only NVTX 3; a no-op unless a profiler
// injects its tool) over every call, cycle, level and colour enqueued on the
// host.  A graph-captured solve carries the ranges of its capture; its
// replays appear as one range per call.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    NvtxRange(const char* fmt, int a, int b = 0, int c = 0) {
        char buf[96];
        snprintf(buf, sizeof buf, fmt, a, b, c);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Logging: CM_LOG=1 prints one line per solve to stderr (size, kind, alpha,
// cycles, first and last energy, convergence, energy rises, wall time of the
// call); CM_LOG=2 adds the energy of every cycle.  Read once per process.
int log_level() {
    static const int level = [] {
        const char* e = getenv("CM_LOG");
        return e ? atoi(e) : 0;
    }();
    return level;
}

void log_solve(const char* what, int i, int H, int W, int kind, float alpha, int L,
               const cm_stats& st, double ms) {
    char label[64];
    if (i >= 0)
        snprintf(label, sizeof label, "%s image %d", what, i);
    else
        snprintf(label, sizeof label, "%s", what);
    fprintf(stderr,
            "[cm] %s %dx%d kind=%d alpha=%g levels=%d cycles=%d E %.9g -> %.9g "
            "converged=%d rises=%d %.3f ms\n",
            label, H, W, kind, alpha, L, st.cycles_run, st.energy_initial, st.energy_final,
            st.converged, st.monotone_violations, ms);
    if (log_level() >= 2)
        for (int c = 0; c < st.trace_len; ++c)
            fprintf(stderr, "[cm]   cycle %d E %.12g\n", c, st.energy_trace[c]);
}

struct cm_ctx {
    int device = 0;
    std::string err;
    float* ubuf = nullptr;
    size_t ubuf_cap = 0;
    double* partials = nullptr;
    size_t partials_cap = 0;
    float* tsums = nullptr;      // coarse path: 32x32 tile sums of S - f
    size_t tsums_cap = 0;
    float* cj = nullptr;         // coarse path: per-block shifts of one level
    size_t cj_cap = 0;
    unsigned int* ticket = nullptr;
    double* E_dev = nullptr;
    double* E_pinned = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_stream2 = nullptr;   // captures the body of the solve loop
    // single-image solve: device stopping state and energy trace, host mirrors
    void* sstate = nullptr;
    void* sstate_host = nullptr;
    double* strace = nullptr;
    double* strace_host = nullptr;
    // batched solve: arena, capture streams/events and the cached batch graph
    unsigned char* arena = nullptr;
    size_t arena_cap = 0;
    std::vector<cudaStream_t> bstreams;
    std::vector<cudaEvent_t> bevents;
    cudaGraphExec_t bgraph = nullptr;
    std::vector<unsigned char> bgraph_key;
    struct Cached {
        bool valid = false;
        GraphKey key;
        cudaGraphExec_t exec = nullptr;
    } sgraph;
    cm::ReconWork* recon = nullptr;   // reconstruction buffers (cm_recon)
};

namespace {

int fail(cm_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

// Host-side fault injection for the tests: with CM_FAULT_ALLOC_LIMIT=<bytes>
// in the environment (read once per process), every scratch allocation of a
// context larger than that fails as cudaErrorMemoryAllocation, so the
// out-of-memory path runs without exhausting the GPU.
size_t fault_alloc_limit() {
    static const size_t lim = [] {
        const char* v = getenv("CM_FAULT_ALLOC_LIMIT");
        return v ? (size_t)strtoull(v, nullptr, 10) : ~(size_t)0;
    }();
    return lim;
}

template <class T>
cudaError_t dev_alloc(T** p, size_t bytes) {
    if (bytes > fault_alloc_limit()) return cudaErrorMemoryAllocation;
    return cudaMalloc((void**)p, bytes);
}

int cuda_fail(cm_ctx* ctx, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? CM_ERR_OOM : CM_ERR_CUDA, m);
}

#define CM_CUDA(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Cached graphs hold scratch pointers: drop them before any reallocation.
void drop_graphs(cm_ctx* ctx) {
    if (ctx->sgraph.exec) cudaGraphExecDestroy(ctx->sgraph.exec);
    ctx->sgraph.exec = nullptr;
    ctx->sgraph.valid = false;
}

int ensure_partials(cm_ctx* ctx, int H, int W) {
    size_t need = cm::energy_partials_needed(H, W);
    if (need <= ctx->partials_cap) return CM_OK;
    drop_graphs(ctx);
    if (ctx->partials) cudaFree(ctx->partials);
    ctx->partials = nullptr;
    ctx->partials_cap = 0;
    CM_CUDA(dev_alloc(&ctx->partials, need * sizeof(double)));
    ctx->partials_cap = need;
    return CM_OK;
}

int ensure_coarse(cm_ctx* ctx, int H, int W) {
    size_t nt = cm::coarse_partials_needed(H, W), nc = cm::coarse_c_needed(H, W);
    if (nt <= ctx->tsums_cap && nc <= ctx->cj_cap) return CM_OK;
    drop_graphs(ctx);
    if (ctx->tsums) cudaFree(ctx->tsums);
    if (ctx->cj) cudaFree(ctx->cj);
    ctx->tsums = nullptr;
    ctx->cj = nullptr;
    ctx->tsums_cap = ctx->cj_cap = 0;
    CM_CUDA(dev_alloc(&ctx->tsums, nt * sizeof(float)));
    CM_CUDA(dev_alloc(&ctx->cj, nc * sizeof(float)));
    ctx->tsums_cap = nt;
    ctx->cj_cap = nc;
    return CM_OK;
}

int ensure_ubuf(cm_ctx* ctx, size_t n) {
    if (n <= ctx->ubuf_cap) return CM_OK;
    drop_graphs(ctx);
    if (ctx->ubuf) cudaFree(ctx->ubuf);
    ctx->ubuf = nullptr;
    ctx->ubuf_cap = 0;
    CM_CUDA(dev_alloc(&ctx->ubuf, n * sizeof(float)));
    ctx->ubuf_cap = n;
    return CM_OK;
}

constexpr int TRACE_SLOTS = 4097;   // energy_trace of cm_stats

int ensure_solve_state(cm_ctx* ctx) {
    if (ctx->sstate) return CM_OK;
    CM_CUDA(dev_alloc(&ctx->sstate, cm::batch_state_bytes()));
    CM_CUDA(cudaMallocHost(&ctx->sstate_host, cm::batch_state_bytes()));
    CM_CUDA(dev_alloc(&ctx->strace, TRACE_SLOTS * sizeof(double)));
    CM_CUDA(cudaMallocHost(&ctx->strace_host, TRACE_SLOTS * sizeof(double)));
    return CM_OK;
}

bool finite_positive(float a) { return isfinite(a) && a > 0.0f; }
// Image sizes the kernels index within (include/cm.h: CM_MAX_SIDE, CM_MAX_PIXELS).
bool dims_ok(int H, int W) {
    return H >= 1 && W >= 1 && H <= CM_MAX_SIDE && W <= CM_MAX_SIDE &&
           (long long)H * W <= CM_MAX_PIXELS;
}
// Curvature kinds: 0 mean, 1 Gaussian (extreme directions), 2 mean, 3 Gaussian
// (Euler fit).
bool valid_kind(int kind) { return kind >= 0 && kind <= 3; }

int check_opts(cm_ctx* ctx, const cm_options& o) {
    if (o.ncolors != 0 && o.ncolors != 2 && o.ncolors != 4 && o.ncolors != 9 && o.ncolors != 16)
        return fail(ctx, CM_ERR_INVALID, "ncolors must be 0, 2, 4, 9 or 16");
    if (o.grid_points < 3 || (o.grid_points % 2) == 0 || o.grid_points > 1025)
        return fail(ctx, CM_ERR_INVALID, "grid_points must be odd, 3..1025");
    if (o.golden_evals < 2 || o.golden_evals > 1024)
        return fail(ctx, CM_ERR_INVALID, "golden_evals must be 2..1024");
    if (o.max_trace < 0 || o.max_trace > 4096) return fail(ctx, CM_ERR_INVALID, "max_trace 0..4096");
    if (o.one_step != 0 && o.one_step != 1) return fail(ctx, CM_ERR_INVALID, "one_step must be 0 or 1");
    if (o.vcycle != 0 && o.vcycle != 1) return fail(ctx, CM_ERR_INVALID, "vcycle must be 0 or 1");
    if (o.coarse_spec < -1 || o.coarse_spec > 1)
        return fail(ctx, CM_ERR_INVALID, "coarse_spec must be -1, 0 or 1");
    if (o.coarse_dmax < 0 || o.coarse_dmax > 4)
        return fail(ctx, CM_ERR_INVALID, "coarse_dmax must be 0 .. 4");
    if (o.block_sides != 0 && o.block_sides != 1)
        return fail(ctx, CM_ERR_INVALID, "block_sides must be 0 or 1");
    if (o.shapes < 0 || o.shapes > 31) return fail(ctx, CM_ERR_INVALID, "shapes must be 0 .. 31");
    if (o.coarse_ncolors != 0 && o.coarse_ncolors != 1 && o.coarse_ncolors != 2 &&
        o.coarse_ncolors != 4 && o.coarse_ncolors != 9 && o.coarse_ncolors != 16)
        return fail(ctx, CM_ERR_INVALID, "coarse_ncolors must be 0, 1, 2, 4, 9 or 16");
    return CM_OK;
}

// Shape class of the block side b of one phase or level: b a power of two or
// one of the paper's sides 2^j - 1, at most 2048; -1 otherwise.
int side_lb(int b) {
    if (b < 1) return -1;
    const int lb = cm::side_class(b);
    if (lb > cm::max_level_log2()) return -1;
    return (b == (1 << lb) || b == (1 << lb) - 1) ? lb : -1;
}

// Levels of the solve: `levels`, or the default for the block-side rule.
int solve_levels(int levels, int H, int W, const cm_options& o) {
    return levels > 0 ? levels : cm::auto_levels(H, W, o.block_sides);
}

// The coarsest level's side is within the kernels' shapes.
bool levels_ok(int L, const cm_options& o) {
    return cm::side_class(cm::level_side(L - 1, o.block_sides)) <= cm::max_level_log2();
}

// Levels of power-of-two side from the coarse threshold on run the coarse
// path (tile sums, search, deferred apply).
bool coarse_side(int b) {
    const int lb = cm::side_class(b);
    return b == (1 << lb) && lb >= cm::coarse_level_log2();
}

cm::PhaseArgs phase_args(const float* S, float* R, const float* f, int H, int W, float alpha,
                         int kind, int b, int colour, const cm_options& o) {
    cm::PhaseArgs a;
    a.S = S;
    a.R = R;
    a.f = f;
    a.H = H;
    a.W = W;
    a.alpha = alpha;
    a.kind = kind;
    a.lb = cm::side_class(b);
    a.bs = b;
    a.ncolors = cm::level_colours(o.ncolors, b, o.coarse_ncolors);
    a.colour = colour;
    a.G = o.grid_points;
    a.K = o.golden_evals;
    a.use_paper = o.paper_candidate;
    a.one_step = o.one_step;
    a.coarse_spec = o.coarse_spec;
    a.coarse_dmax = o.coarse_dmax;
    a.shapes = o.shapes;
    a.c_out = nullptr;
    return a;
}

// Enqueue one level of block side b (all colours) from state S into R.
// Levels below the coarse threshold, and levels of odd side, run one phase
// kernel per colour; coarse levels run the tile-sum / search / apply
// sequence.  c_out (nullable) receives every block's shift.  read_colour
// (phase kernels of b >= 2): -1 as the colour, or 0 with R == S to run the
// level in place (cm::in_place_ok).
cudaError_t enqueue_level(float* tsums, float* cj, const float* S, float* R, const float* f,
                          int H, int W, float alpha, int kind, int b, const cm_options& o,
                          float* c_out, const int* active, cudaStream_t st,
                          bool sums_ready = false, int read_colour = -1) {
    NvtxRange level("level b=%d", b);
    if (coarse_side(b)) {
        cm::PhaseArgs a = phase_args(S, R, f, H, W, alpha, kind, b, 0, o);
        a.c_out = c_out;
        a.active = active;
        return cm::launch_level_coarse(a, tsums, cj, st, sums_ready);
    }
    const int nc = cm::level_colours(o.ncolors, b, o.coarse_ncolors);
    for (int k = 0; k < nc; ++k) {
        NvtxRange colour("colour %d", k);
        cm::PhaseArgs a = phase_args(S, R, f, H, W, alpha, kind, b, k, o);
        a.c_out = c_out;
        a.active = active;
        a.read_colour = read_colour;
        cudaError_t e = cm::launch_phase(a, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Level steps of one cycle: levels 0 .. L-1 (the half V-cycle of Alg. 3),
// with vcycle also back up, L-2 .. 0.
int level_steps(int L, const cm_options& o) { return o.vcycle ? 2 * L - 1 : L; }
int level_at(int step, int L) { return step < L ? step : 2 * L - 2 - step; }

// Enqueue one cycle starting from buffer X (other buffer Y), then the energy
// of the final state.  Levels of b >= 2 whose colouring keeps same-coloured
// blocks out of each other's read windows (cm::in_place_ok) run in place:
// a phase then reads the state being updated, which holds the new values of
// the earlier colours and the old values of the rest, exactly what the
// S / R pair of Alg. 1's snapshot gives, without the per-pixel colour test.
// Every other level reads S and writes R, and the two swap.  With end_in_x
// the state always ends in X: an odd count of swaps runs its last level in
// place when that level is on the coarse path (whose phases only read S and
// whose final apply writes each pixel from itself), else copies Y to X.
cudaError_t enqueue_cycle(cm_ctx* ctx, float* X, float* Y, const float* f, int H, int W,
                          float alpha, int kind, int levels, const cm_options& o,
                          cudaStream_t st, bool end_in_x = false, bool* ended_in_y = nullptr) {
    float* S = X;
    float* R = Y;
    const int nsteps = level_steps(levels, o);
    bool sums = false;   // tile sums of the current state already in ctx->tsums
    for (int step = 0; step < nsteps; ++step) {
        const int b = cm::level_side(level_at(step, levels), o.block_sides);
        const bool coarse = coarse_side(b);
        const bool fine_in_place =
            !coarse && cm::in_place_ok(b, cm::level_colours(o.ncolors, b, o.coarse_ncolors));
        const bool in_place =
            fine_in_place || (end_in_x && step == nsteps - 1 && S == X && coarse);
        float* out = in_place ? S : R;
        cudaError_t e = enqueue_level(ctx->tsums, ctx->cj, S, out, f, H, W, alpha, kind, b, o,
                                      nullptr, nullptr, st, sums, fine_in_place ? 0 : -1);
        sums = coarse;
        if (e != cudaSuccess) return e;
        if (!in_place) {
            float* t = S;
            S = R;
            R = t;
        }
    }
    if (end_in_x && S != X) {
        cudaError_t e = cudaMemcpyAsync(X, S, (size_t)H * W * sizeof(float),
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        S = X;
    }
    if (ended_in_y) *ended_in_y = S != X;
    return cm::launch_energy(S, f, H, W, alpha, kind, ctx->partials, ctx->ticket, ctx->E_dev, st);
}

// Capture the whole solve of u (in place, scratch Y) as one graph: the
// initial energy, the state's initialisation, and a WHILE node around one
// cycle plus the stopping test.
cudaError_t capture_solve(cm_ctx* ctx, float* u, float* Y, const float* f, int H, int W,
                          float alpha, int kind, int levels, const cm_options& o, double tol,
                          int cycles, int trace_cap, cudaGraphExec_t* exec) {
    cm::ImgDev* state = static_cast<cm::ImgDev*>(ctx->sstate);
    cudaStream_t s1 = ctx->cap_stream, s2 = ctx->cap_stream2;
    cudaError_t e = cudaStreamBeginCapture(s1, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    bool body_open = false;
    cudaGraph_t g = nullptr;
    cudaStreamCaptureStatus cs;
    cudaGraphConditionalHandle h = 0;
    do {
        if ((e = cudaStreamGetCaptureInfo(s1, &cs, nullptr, &g)) != cudaSuccess) break;
        if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, 0)) != cudaSuccess) break;
        if ((e = cm::launch_energy(u, f, H, W, alpha, kind, ctx->partials, ctx->ticket,
                                   ctx->E_dev, s1)) != cudaSuccess)
            break;
        if ((e = cm::launch_solve_init(state, ctx->E_dev, cycles, ctx->strace, h, s1)) !=
            cudaSuccess)
            break;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        if ((e = cudaStreamGetCaptureInfo(s1, &cs, nullptr, nullptr, &deps, nullptr, &nd)) !=
            cudaSuccess)
            break;
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t wnode;
        if ((e = cudaGraphAddNode(&wnode, g, deps, nullptr, nd, &cp)) != cudaSuccess) break;
        if ((e = cudaStreamUpdateCaptureDependencies(s1, &wnode, nullptr, 1,
                                                     cudaStreamSetCaptureDependencies)) !=
            cudaSuccess)
            break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            break;
        body_open = true;
        if ((e = enqueue_cycle(ctx, u, Y, f, H, W, alpha, kind, levels, o, s2, true)) !=
            cudaSuccess)
            break;
        e = cm::launch_solve_stop(state, ctx->E_dev, tol, cycles, ctx->strace, trace_cap, h, s2);
    } while (false);
    if (body_open) {
        cudaGraph_t b2 = nullptr;
        cudaError_t ee = cudaStreamEndCapture(s2, &b2);
        if (e == cudaSuccess) e = ee;
    }
    cudaGraph_t done = nullptr;
    cudaError_t ee = cudaStreamEndCapture(s1, &done);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, done, 0);
    if (done) cudaGraphDestroy(done);
    return e;
}

}  // namespace

// Shared tail of cm_recon and cm_recon_ct: levels from the options, the
// context's reconstruction buffers, the run and its status.
int run_recon(cm_ctx* ctx, cm::ReconArgs& a, int levels, const cm_options& o, void* stream,
              const char* name) {
    NvtxRange range(a.op == cm::RECON_MRI ? "cm_recon %dx%d" : "cm_recon_ct %dx%d", a.H, a.W);
    const int L = solve_levels(levels, a.H, a.W, o);
    if (!levels_ok(L, o)) return fail(ctx, CM_ERR_INVALID, std::string(name) + ": too many levels");
    CM_CUDA(cudaSetDevice(ctx->device));
    if (!ctx->recon) ctx->recon = cm::recon_work_create();
    a.levels = L;
    a.sides = o.block_sides;
    a.ncolors = o.ncolors;
    const char* msg = "";
    const int rc = cm::recon_run(ctx->recon, a, (cudaStream_t)stream, &msg);
    if (rc == 1) return fail(ctx, CM_ERR_INVALID, std::string(name) + ": " + msg);
    if (rc == 3) return fail(ctx, CM_ERR_OOM, std::string(name) + ": " + msg);
    if (rc) return fail(ctx, CM_ERR_CUDA, std::string(name) + ": " + msg);
    return CM_OK;
}

extern "C" {

int cm_options_default(cm_options* o) {
    if (!o) return CM_ERR_INVALID;
    o->ncolors = 4;
    o->grid_points = 5;
    o->golden_evals = 6;
    o->paper_candidate = 1;
    o->use_graph = 1;
    o->max_trace = 4096;
    o->one_step = 0;
    o->vcycle = 0;
    o->coarse_spec = -1;
    o->coarse_dmax = 0;
    o->shapes = 0;
    o->coarse_ncolors = 0;
    o->block_sides = 0;
    return CM_OK;
}

int cm_auto_levels(int H, int W) {
    int m = H < W ? H : W;
    int L = 1, b = 1;
    while (2 * b <= m / 2) {
        b *= 2;
        ++L;
    }
    return L;
}

int cm_create(cm_ctx** out, int device) {
    if (!out) return CM_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return CM_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return CM_ERR_CUDA;
    cm_ctx* ctx = new cm_ctx();
    ctx->device = device;
    cudaError_t e = dev_alloc(&ctx->ticket, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(ctx->ticket, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = dev_alloc(&ctx->E_dev, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->E_pinned, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cm::coarse_setup();
    if (e == cudaSuccess) e = cm::fft_setup();
    if (e != cudaSuccess) {
        cm_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? CM_ERR_OOM : CM_ERR_CUDA;
    }
    *out = ctx;
    return CM_OK;
}

void cm_destroy(cm_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->sgraph.exec) cudaGraphExecDestroy(ctx->sgraph.exec);
    if (ctx->sstate) cudaFree(ctx->sstate);
    if (ctx->sstate_host) cudaFreeHost(ctx->sstate_host);
    if (ctx->strace) cudaFree(ctx->strace);
    if (ctx->strace_host) cudaFreeHost(ctx->strace_host);
    if (ctx->cap_stream2) cudaStreamDestroy(ctx->cap_stream2);
    if (ctx->ubuf) cudaFree(ctx->ubuf);
    if (ctx->partials) cudaFree(ctx->partials);
    if (ctx->tsums) cudaFree(ctx->tsums);
    if (ctx->cj) cudaFree(ctx->cj);
    if (ctx->ticket) cudaFree(ctx->ticket);
    if (ctx->E_dev) cudaFree(ctx->E_dev);
    if (ctx->E_pinned) cudaFreeHost(ctx->E_pinned);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
    for (auto s : ctx->bstreams) cudaStreamDestroy(s);
    for (auto e : ctx->bevents) cudaEventDestroy(e);
    if (ctx->arena) cudaFree(ctx->arena);
    cm::recon_work_destroy(ctx->recon);
    delete ctx;
}

const char* cm_last_error(const cm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int cm_energy(cm_ctx* ctx, const float* u, const float* f, int H, int W, float alpha, int kind,
              double* E_host, void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    if (!u || !f || !E_host || !dims_ok(H, W) || !finite_positive(alpha) || !valid_kind(kind))
        return fail(ctx, CM_ERR_INVALID, "cm_energy: invalid argument");
    CM_CUDA(cudaSetDevice(ctx->device));
    int rc = ensure_partials(ctx, H, W);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CM_CUDA(cm::launch_energy(u, f, H, W, alpha, kind, ctx->partials, ctx->ticket, ctx->E_dev, st));
    CM_CUDA(cudaMemcpyAsync(ctx->E_pinned, ctx->E_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    CM_CUDA(cudaStreamSynchronize(st));
    *E_host = ctx->E_pinned[0];
    if (!isfinite(*E_host)) return fail(ctx, CM_ERR_NUMERIC, "cm_energy: non-finite energy");
    return CM_OK;
}

int cm_curvature(cm_ctx* ctx, const float* u, int H, int W, int kind, float* out, void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    if (!u || !out || !dims_ok(H, W) || !valid_kind(kind))
        return fail(ctx, CM_ERR_INVALID, "cm_curvature: invalid argument");
    CM_CUDA(cudaSetDevice(ctx->device));
    CM_CUDA(cm::launch_curvature(u, H, W, kind, out, (cudaStream_t)stream));
    return CM_OK;
}

int cm_phase(cm_ctx* ctx, const float* S, float* R, const float* f, int H, int W, float alpha,
             int kind, int b, int colour, const cm_options* opts, float* c_out, void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    cm_options o;
    cm_options_default(&o);
    if (opts) o = *opts;
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    if (!S || !R || !f || R == S || R == f || !dims_ok(H, W) || !finite_positive(alpha) ||
        !valid_kind(kind))
        return fail(ctx, CM_ERR_INVALID, "cm_phase: invalid argument");
    if (side_lb(b) < 0)
        return fail(ctx, CM_ERR_INVALID, "cm_phase: b must be 2^j or 2^j - 1, at most 2048");
    if (colour < 0 || colour >= cm::level_colours(o.ncolors, b, o.coarse_ncolors))
        return fail(ctx, CM_ERR_INVALID, "cm_phase: bad colour");
    CM_CUDA(cudaSetDevice(ctx->device));
    cm::PhaseArgs a = phase_args(S, R, f, H, W, alpha, kind, b, colour, o);
    a.c_out = c_out;
    CM_CUDA(cm::launch_phase(a, (cudaStream_t)stream));
    return CM_OK;
}

int cm_level(cm_ctx* ctx, const float* S, float* R, const float* f, int H, int W, float alpha,
             int kind, int b, const cm_options* opts, float* c_out, void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    cm_options o;
    cm_options_default(&o);
    if (opts) o = *opts;
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    if (!S || !R || !f || R == S || R == f || !dims_ok(H, W) || !finite_positive(alpha) ||
        !valid_kind(kind))
        return fail(ctx, CM_ERR_INVALID, "cm_level: invalid argument");
    if (side_lb(b) < 0)
        return fail(ctx, CM_ERR_INVALID, "cm_level: b must be 2^j or 2^j - 1, at most 2048");
    CM_CUDA(cudaSetDevice(ctx->device));
    rc = ensure_coarse(ctx, H, W);
    if (rc) return rc;
    CM_CUDA(enqueue_level(ctx->tsums, ctx->cj, S, R, f, H, W, alpha, kind, b, o, c_out, nullptr,
                          (cudaStream_t)stream));
    return CM_OK;
}

static int solve_impl(cm_ctx* ctx, const float* f, int H, int W, float alpha, int kind,
                      int levels, int cycles, double tol, const float* u0, float* u_out,
                      const cm_options* opts, cm_stats* stats, void* stream);

int cm_solve(cm_ctx* ctx, const float* f, int H, int W, float alpha, int kind, int levels,
             int cycles, double tol, const float* u0, float* u_out, const cm_options* opts,
             cm_stats* stats, void* stream) {
    NvtxRange range("cm_solve %dx%d", H, W);
    if (!log_level())
        return solve_impl(ctx, f, H, W, alpha, kind, levels, cycles, tol, u0, u_out, opts, stats,
                          stream);
    cm_stats local;
    cm_stats* st = stats ? stats : &local;
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = solve_impl(ctx, f, H, W, alpha, kind, levels, cycles, tol, u0, u_out, opts,
                              st, stream);
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc == CM_OK || rc == CM_NOT_CONVERGED)
        log_solve("cm_solve", -1, H, W, kind, alpha, st->levels, *st, ms);
    else
        fprintf(stderr, "[cm] cm_solve %dx%d: status %d (%s)\n", H, W, rc, cm_last_error(ctx));
    return rc;
}

static int solve_impl(cm_ctx* ctx, const float* f, int H, int W, float alpha, int kind,
                      int levels, int cycles, double tol, const float* u0, float* u_out,
                      const cm_options* opts, cm_stats* stats, void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    cm_options o;
    cm_options_default(&o);
    if (opts) o = *opts;
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    if (!f || !u_out || u_out == f || !dims_ok(H, W) || !finite_positive(alpha) ||
        !valid_kind(kind) || levels < 0 || cycles < 0 || !(tol >= 0.0) || !isfinite(tol))
        return fail(ctx, CM_ERR_INVALID, "cm_solve: invalid argument");
    const int L = solve_levels(levels, H, W, o);
    if (!levels_ok(L, o)) return fail(ctx, CM_ERR_INVALID, "cm_solve: too many levels");
    CM_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)H * W;
    rc = ensure_partials(ctx, H, W);
    if (rc) return rc;
    rc = ensure_ubuf(ctx, N);
    if (rc) return rc;
    rc = ensure_coarse(ctx, H, W);
    if (rc) return rc;
    float* bufs[2] = {u_out, ctx->ubuf};
    if (u0 && u0 != u_out)
        CM_CUDA(cudaMemcpyAsync(u_out, u0, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    else if (!u0)
        CM_CUDA(cudaMemcpyAsync(u_out, f, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (o.use_graph) {
        // the whole solve as one graph: loop and stopping test on the device
        rc = ensure_solve_state(ctx);
        if (rc) return rc;
        const int trace_cap = std::min(cycles, o.max_trace);
        GraphKey key;
        memset(&key, 0, sizeof(key));
        key.S = u_out;
        key.R = ctx->ubuf;
        key.f = f;
        key.H = H;
        key.W = W;
        key.kind = kind;
        key.levels = L;
        key.ncolors = o.ncolors;
        key.G = o.grid_points;
        key.K = o.golden_evals;
        key.use_paper = o.paper_candidate;
        key.one_step = o.one_step;
        key.vcycle = o.vcycle;
        key.coarse_spec = o.coarse_spec;
        key.coarse_dmax = o.coarse_dmax;
        key.block_sides = o.block_sides;
        key.coarse_ncolors = o.coarse_ncolors;
        key.shapes = o.shapes;
        key.alpha = alpha;
        key.tol = tol;
        key.cycles = cycles;
        key.trace_cap = trace_cap;
        auto& slot = ctx->sgraph;
        if (!slot.valid || !(slot.key == key)) {
            drop_graphs(ctx);
            cudaError_t ce = capture_solve(ctx, u_out, ctx->ubuf, f, H, W, alpha, kind, L, o, tol,
                                           cycles, trace_cap, &slot.exec);
            if (ce != cudaSuccess) {
                slot.exec = nullptr;
                return cuda_fail(ctx, ce, "capture solve graph");
            }
            slot.key = key;
            slot.valid = true;
        }
        CM_CUDA(cudaGraphLaunch(slot.exec, st));
        CM_CUDA(cudaMemcpyAsync(ctx->sstate_host, ctx->sstate, cm::batch_state_bytes(),
                                cudaMemcpyDeviceToHost, st));
        CM_CUDA(cudaStreamSynchronize(st));
        int ncyc = 0, conv = 0, viol = 0, numeric = 0, act = 0;
        double E = 0.0;
        cm::batch_read_state(ctx->sstate_host, &ncyc, &conv, &viol, &E, &numeric, &act);
        const int tl = std::min(ncyc, trace_cap) + 1;
        CM_CUDA(cudaMemcpyAsync(ctx->strace_host, ctx->strace, tl * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
        CM_CUDA(cudaStreamSynchronize(st));
        if (stats) {
            memset(stats, 0, sizeof(*stats));
            stats->levels = L;
            stats->energy_initial = ctx->strace_host[0];
            stats->trace_len = tl;
            memcpy(stats->energy_trace, ctx->strace_host, tl * sizeof(double));
            stats->cycles_run = ncyc;
            stats->converged = conv;
            stats->monotone_violations = viol;
            stats->energy_final = ncyc > 0 ? E : ctx->strace_host[0];
        }
        if (numeric)
            return fail(ctx, CM_ERR_NUMERIC, ncyc == 0 ? "cm_solve: non-finite initial energy"
                                                       : "cm_solve: non-finite energy");
        if (tol > 0.0 && !conv) return fail(ctx, CM_NOT_CONVERGED, "cm_solve: cycle cap reached");
        return CM_OK;
    }
    // host loop (use_graph = 0): one cycle at a time, 8 bytes read back per cycle
    CM_CUDA(cm::launch_energy(u_out, f, H, W, alpha, kind, ctx->partials, ctx->ticket, ctx->E_dev, st));
    CM_CUDA(cudaMemcpyAsync(ctx->E_pinned, ctx->E_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    CM_CUDA(cudaStreamSynchronize(st));
    double Eprev = ctx->E_pinned[0];
    if (!isfinite(Eprev)) return fail(ctx, CM_ERR_NUMERIC, "cm_solve: non-finite initial energy");
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->levels = L;
        stats->energy_initial = Eprev;
        stats->energy_trace[0] = Eprev;
        stats->trace_len = 1;
    }
    int cur = 0, l = 0, conv = 0, viol = 0;
    while (l < cycles) {
        NvtxRange cyc("cycle %d", l + 1);
        float* X = bufs[cur];
        float* Y = bufs[cur ^ 1];
        bool in_y = false;
        CM_CUDA(enqueue_cycle(ctx, X, Y, f, H, W, alpha, kind, L, o, st, false, &in_y));
        if (in_y) cur ^= 1;
        CM_CUDA(cudaMemcpyAsync(ctx->E_pinned, ctx->E_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
        CM_CUDA(cudaStreamSynchronize(st));
        ++l;
        double E = ctx->E_pinned[0];
        if (!isfinite(E)) return fail(ctx, CM_ERR_NUMERIC, "cm_solve: non-finite energy");
        if (E > Eprev) ++viol;
        if (stats && stats->trace_len <= o.max_trace) stats->energy_trace[stats->trace_len++] = E;
        bool stop = tol > 0.0 && fabs(E - Eprev) <= tol * fabs(E);
        Eprev = E;
        if (stop) {
            conv = 1;
            break;
        }
    }
    if (cur != 0)
        CM_CUDA(cudaMemcpyAsync(u_out, bufs[cur], N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    CM_CUDA(cudaStreamSynchronize(st));
    if (stats) {
        stats->cycles_run = l;
        stats->converged = conv;
        stats->monotone_violations = viol;
        stats->energy_final = Eprev;
    }
    if (tol > 0.0 && !conv) return fail(ctx, CM_NOT_CONVERGED, "cm_solve: cycle cap reached");
    return CM_OK;
}


// ---------------------------------------------------------------------------
// Learned warm start.

int cm_warmstart(cm_ctx* ctx, cm_net* net, const float* f, int N, int H, int W, float* u0_out,
                 int check_energy, float alpha, int kind, int* used_host, void* stream) {
    NvtxRange range("cm_warmstart %d x %dx%d", N, H, W);
    if (!ctx) return CM_ERR_INVALID;
    if (!net || !f || !u0_out || u0_out == f || N < 1 || !dims_ok(H, W) ||
        (check_energy && (!finite_positive(alpha) || !valid_kind(kind))))
        return fail(ctx, CM_ERR_INVALID, "cm_warmstart: invalid argument");
    CM_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    cm::cnn::Net* nn = reinterpret_cast<cm::cnn::Net*>(net);
    int rc = cm::cnn::net_forward(nn, f, N, H, W, u0_out, st);
    if (rc) return fail(ctx, rc, std::string("cm_warmstart: ") + cm::cnn::net_error(nn));
    const size_t npx = (size_t)H * W;
    if (check_energy) {
        rc = ensure_partials(ctx, H, W);
        if (rc) return rc;
        for (int n = 0; n < N; ++n) {
            const float* fi = f + n * npx;
            float* ui = u0_out + n * npx;
            // the sweep's energy decides on the network's output: keep u0 only if F(u0) <= F(f)
            CM_CUDA(cm::launch_energy(ui, fi, H, W, alpha, kind, ctx->partials, ctx->ticket,
                                      &ctx->E_dev[0], st));
            CM_CUDA(cm::launch_energy(fi, fi, H, W, alpha, kind, ctx->partials, ctx->ticket,
                                      &ctx->E_dev[1], st));
            CM_CUDA(cudaMemcpyAsync(ctx->E_pinned, ctx->E_dev, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
            CM_CUDA(cudaStreamSynchronize(st));
            if (n == 0) {
                rc = cm::cnn::net_status(nn);
                if (rc) return fail(ctx, rc, std::string("cm_warmstart: ") + cm::cnn::net_error(nn));
            }
            const bool keep = isfinite(ctx->E_pinned[0]) && ctx->E_pinned[0] <= ctx->E_pinned[1];
            if (!keep)
                CM_CUDA(cudaMemcpyAsync(ui, fi, npx * sizeof(float), cudaMemcpyDeviceToDevice, st));
            if (used_host) used_host[n] = keep ? 1 : 0;
        }
    } else if (used_host) {
        for (int n = 0; n < N; ++n) used_host[n] = 1;
    }
    return CM_OK;
}

// ---------------------------------------------------------------------------
// Batched solve.

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct ImgLayout {
    size_t ubuf, partials, ticket, tsums, cj, trace;
    int L;
};

}  // namespace

static int solve_batched_impl(cm_ctx* ctx, int n, const float* const* f, const int* H,
                              const int* W, const float* alpha, const int* kind, int levels,
                              int cycles, double tol, const float* const* u0,
                              float* const* u_out, const cm_options* opts, cm_stats* stats,
                              void* stream);

int cm_solve_batched(cm_ctx* ctx, int n, const float* const* f, const int* H, const int* W,
                     const float* alpha, const int* kind, int levels, int cycles, double tol,
                     const float* const* u0, float* const* u_out, const cm_options* opts,
                     cm_stats* stats, void* stream) {
    NvtxRange range("cm_solve_batched %d images", n);
    if (!log_level() || n < 1 || !H || !W || !alpha || !kind)
        return solve_batched_impl(ctx, n, f, H, W, alpha, kind, levels, cycles, tol, u0, u_out,
                                  opts, stats, stream);
    std::vector<cm_stats> local(stats ? 0 : (size_t)n);
    cm_stats* st = stats ? stats : local.data();
    const auto t0 = std::chrono::steady_clock::now();
    const int rc = solve_batched_impl(ctx, n, f, H, W, alpha, kind, levels, cycles, tol, u0,
                                      u_out, opts, st, stream);
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc == CM_OK || rc == CM_NOT_CONVERGED)
        for (int i = 0; i < n; ++i)
            log_solve("cm_solve_batched", i, H[i], W[i], kind[i], alpha[i], st[i].levels, st[i],
                      ms);
    else
        fprintf(stderr, "[cm] cm_solve_batched: status %d (%s)\n", rc, cm_last_error(ctx));
    return rc;
}

static int solve_batched_impl(cm_ctx* ctx, int n, const float* const* f, const int* H,
                              const int* W, const float* alpha, const int* kind, int levels,
                              int cycles, double tol, const float* const* u0,
                              float* const* u_out, const cm_options* opts, cm_stats* stats,
                              void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    cm_options o;
    cm_options_default(&o);
    if (opts) o = *opts;
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    if (n < 1 || !f || !H || !W || !alpha || !kind || !u_out || levels < 0 || cycles < 0 ||
        !(tol >= 0.0) || !isfinite(tol))
        return fail(ctx, CM_ERR_INVALID, "cm_solve_batched: invalid argument");
    for (int i = 0; i < n; ++i) {
        if (!f[i] || !u_out[i] || u_out[i] == f[i] || !dims_ok(H[i], W[i]) ||
            !finite_positive(alpha[i]) || !valid_kind(kind[i]))
            return fail(ctx, CM_ERR_INVALID, "cm_solve_batched: invalid image " + std::to_string(i));
        const int L = solve_levels(levels, H[i], W[i], o);
        if (!levels_ok(L, o))
            return fail(ctx, CM_ERR_INVALID, "cm_solve_batched: too many levels");
    }
    CM_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int trace_cap = std::min(cycles, o.max_trace);
    // arena: per-image scratch, then the state array and initial energies
    std::vector<ImgLayout> lay(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const size_t N = (size_t)H[i] * W[i];
        ImgLayout& L = lay[i];
        L.L = solve_levels(levels, H[i], W[i], o);
        L.ubuf = off; off = align256(off + N * sizeof(float));
        L.partials = off; off = align256(off + cm::energy_partials_needed(H[i], W[i]) * sizeof(double));
        L.ticket = off; off = align256(off + sizeof(unsigned int));
        L.tsums = off; off = align256(off + cm::coarse_partials_needed(H[i], W[i]) * sizeof(float));
        L.cj = off; off = align256(off + cm::coarse_c_needed(H[i], W[i]) * sizeof(float));
        L.trace = off; off = align256(off + (size_t)(trace_cap + 1) * sizeof(double));
    }
    const size_t state_off = off;
    const size_t sb = cm::batch_state_bytes();
    off = align256(off + (size_t)n * sb);
    const size_t e0_off = off;
    off = align256(off + (size_t)n * sizeof(double));
    const size_t enow_off = off;
    off = align256(off + (size_t)n * sizeof(double));
    if (off > ctx->arena_cap) {
        if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
        ctx->bgraph = nullptr;
        ctx->bgraph_key.clear();
        if (ctx->arena) cudaFree(ctx->arena);
        ctx->arena = nullptr;
        ctx->arena_cap = 0;
        CM_CUDA(dev_alloc(&ctx->arena, off));
        ctx->arena_cap = off;
    }
    unsigned char* A = ctx->arena;
    auto state_ptr = [&](int i) { return (cm::ImgDev*)(A + state_off + (size_t)i * sb); };
    auto active_ptr = [&](int i) { return (const int*)(A + state_off + (size_t)i * sb + cm::batch_active_offset()); };
    double* E0 = (double*)(A + e0_off);
    double* Enow = (double*)(A + enow_off);
    // initial state u_0 and energies
    for (int i = 0; i < n; ++i) {
        const size_t N = (size_t)H[i] * W[i];
        const float* src = (u0 && u0[i]) ? u0[i] : f[i];
        if (src != u_out[i])
            CM_CUDA(cudaMemcpyAsync(u_out[i], src, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
        CM_CUDA(cudaMemsetAsync(A + lay[i].ticket, 0, sizeof(unsigned int), st));
        CM_CUDA(cm::launch_energy(u_out[i], f[i], H[i], W[i], alpha[i], kind[i],
                                  (double*)(A + lay[i].partials), (unsigned int*)(A + lay[i].ticket),
                                  &E0[i], st));
    }
    CM_CUDA(cm::launch_batch_init(state_ptr(0), E0, n, cycles, st));
    // the batch-cycle graph (cached for identical batches)
    std::vector<unsigned char> key;
    auto put = [&](const void* p, size_t b) {
        const unsigned char* c = (const unsigned char*)p;
        key.insert(key.end(), c, c + b);
    };
    put(&n, sizeof(n));
    put(&o, sizeof(o));
    put(&levels, sizeof(levels));
    put(&cycles, sizeof(cycles));
    put(&tol, sizeof(tol));
    put(&ctx->arena, sizeof(ctx->arena));
    for (int i = 0; i < n; ++i) {
        put(&f[i], sizeof(f[i]));
        put(&u_out[i], sizeof(u_out[i]));
        put(&H[i], sizeof(int));
        put(&W[i], sizeof(int));
        put(&alpha[i], sizeof(float));
        put(&kind[i], sizeof(int));
    }
    if (!ctx->bgraph || ctx->bgraph_key != key) {
        if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
        ctx->bgraph = nullptr;
        ctx->bgraph_key.clear();
        while ((int)ctx->bstreams.size() < n) {
            cudaStream_t s2;
            CM_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
            ctx->bstreams.push_back(s2);
        }
        while ((int)ctx->bevents.size() < n + 1) {
            cudaEvent_t e2;
            CM_CUDA(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
            ctx->bevents.push_back(e2);
        }
        // the whole batched solve as one graph: a conditional WHILE node (its
        // condition reset to 1 at every launch) around one cycle of every
        // image, the last kernel of which sets the condition to "some image is
        // still active"; every image stops itself at the cycle cap.
        cudaStream_t cs = ctx->cap_stream;
        cudaGraph_t top = nullptr;
        CM_CUDA(cudaGraphCreate(&top, 0));
        cudaGraphConditionalHandle h = 0;
        cudaGraph_t body = nullptr;
        {
            cudaError_t e1 = cudaGraphConditionalHandleCreate(&h, top, 1, cudaGraphCondAssignDefault);
            cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t wnode;
            if (e1 == cudaSuccess) e1 = cudaGraphAddNode(&wnode, top, nullptr, nullptr, 0, &cp);
            if (e1 != cudaSuccess) {
                cudaGraphDestroy(top);
                return cuda_fail(ctx, e1, "batch loop node");
            }
            body = cp.conditional.phGraph_out[0];
        }
        {
            cudaError_t e1 = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                                           cudaStreamCaptureModeThreadLocal);
            if (e1 != cudaSuccess) {
                cudaGraphDestroy(top);
                return cuda_fail(ctx, e1, "capture batch cycle");
            }
        }
        cudaError_t ce = cudaEventRecord(ctx->bevents[n], cs);
        for (int i = 0; i < n && ce == cudaSuccess; ++i) {
            cudaStream_t si = ctx->bstreams[i];
            ce = cudaStreamWaitEvent(si, ctx->bevents[n], 0);
            const ImgLayout& L = lay[i];
            float* X = u_out[i];
            float* Y = (float*)(A + L.ubuf);
            float* Sb = X;
            float* Rb = Y;
            const int nsteps = level_steps(L.L, o);
            bool sums = false;
            for (int step = 0; step < nsteps && ce == cudaSuccess; ++step) {
                const int b = cm::level_side(level_at(step, L.L), o.block_sides);
                // in place as in enqueue_cycle
                const bool ip = !coarse_side(b) &&
                                cm::in_place_ok(b, cm::level_colours(o.ncolors, b, o.coarse_ncolors));
                ce = enqueue_level((float*)(A + L.tsums), (float*)(A + L.cj), Sb, ip ? Sb : Rb,
                                   f[i], H[i], W[i], alpha[i], kind[i], b, o, nullptr,
                                   active_ptr(i), si, sums, ip ? 0 : -1);
                sums = coarse_side(b);
                if (!ip) {
                    float* t = Sb;
                    Sb = Rb;
                    Rb = t;
                }
            }
            const size_t N = (size_t)H[i] * W[i];
            if (ce == cudaSuccess && Sb != X) ce = cm::launch_batch_copy(Sb, X, N, active_ptr(i), si);
            if (ce == cudaSuccess)
                ce = cm::launch_energy(X, f[i], H[i], W[i], alpha[i], kind[i],
                                       (double*)(A + L.partials), (unsigned int*)(A + L.ticket),
                                       &Enow[i], si, active_ptr(i));
            if (ce == cudaSuccess)
                ce = cm::launch_batch_stop(state_ptr(i), &Enow[i], tol, cycles,
                                           (double*)(A + L.trace), trace_cap, si);
            if (ce == cudaSuccess) ce = cudaEventRecord(ctx->bevents[i], si);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, ctx->bevents[i], 0);
        }
        if (ce == cudaSuccess)
            ce = cm::launch_batch_any(state_ptr(0), n, h, cs);
        cudaGraph_t g = nullptr;
        cudaError_t ee = cudaStreamEndCapture(cs, &g);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            cudaGraphDestroy(top);
            return cuda_fail(ctx, ce != cudaSuccess ? ce : ee, "capture batch cycle");
        }
        cudaError_t ie = cudaGraphInstantiate(&ctx->bgraph, top, 0);
        cudaGraphDestroy(top);
        if (ie != cudaSuccess) return cuda_fail(ctx, ie, "batch graph instantiate");
        ctx->bgraph_key = key;
    }
    // one launch runs every cycle of every image; the state is read once
    CM_CUDA(cudaGraphLaunch(ctx->bgraph, st));
    std::vector<unsigned char> host_state((size_t)n * sb);
    CM_CUDA(cudaMemcpyAsync(host_state.data(), state_ptr(0), (size_t)n * sb,
                            cudaMemcpyDeviceToHost, st));
    std::vector<double> e0h(n);
    CM_CUDA(cudaMemcpyAsync(e0h.data(), E0, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CM_CUDA(cudaStreamSynchronize(st));
    int status = CM_OK;
    for (int i = 0; i < n; ++i) {
        int c, cv, v, ne, act;
        double E;
        cm::batch_read_state(host_state.data() + (size_t)i * sb, &c, &cv, &v, &E, &ne, &act);
        if (ne) status = CM_ERR_NUMERIC;
        else if (tol > 0.0 && !cv && status == CM_OK) status = CM_NOT_CONVERGED;
        if (stats) {
            cm_stats& s2 = stats[i];
            memset(&s2, 0, sizeof(s2));
            s2.cycles_run = c;
            s2.converged = cv;
            s2.monotone_violations = v;
            s2.levels = lay[i].L;
            s2.energy_initial = e0h[i];
            s2.energy_final = c > 0 ? E : e0h[i];
            const int tl = std::min(c, trace_cap);
            s2.energy_trace[0] = e0h[i];
            if (tl > 0)
                CM_CUDA(cudaMemcpy(&s2.energy_trace[1], (double*)(A + lay[i].trace) + 1,
                                   (size_t)tl * sizeof(double), cudaMemcpyDeviceToHost));
            s2.trace_len = tl + 1;
        }
    }
    if (status == CM_ERR_NUMERIC) return fail(ctx, status, "cm_solve_batched: non-finite energy");
    if (status == CM_NOT_CONVERGED) return fail(ctx, status, "cm_solve_batched: cycle cap reached");
    return CM_OK;
}

int cm_recon(cm_ctx* ctx, const float* kspace, const unsigned char* mask, int H, int W,
             float alpha, int kind, int levels, int cycles, int cg_iters, const float* u0,
             float* u_out, const cm_options* opts, double* trace_host, void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    cm_options o;
    cm_options_default(&o);
    if (opts) o = *opts;
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    if (!kspace || !mask || !u_out || !dims_ok(H, W) || !finite_positive(alpha) ||
        !valid_kind(kind) || levels < 0 || cycles < 0 || cycles > 100000 || cg_iters < 1 ||
        cg_iters > 1000 || (const void*)u_out == (const void*)kspace)
        return fail(ctx, CM_ERR_INVALID, "cm_recon: invalid argument");
    cm::ReconArgs a;
    a.op = cm::RECON_MRI;
    a.kspace = (const float2*)kspace;
    a.mask = mask;
    a.sino = nullptr;
    a.n_angles = 0;
    a.H = H;
    a.W = W;
    a.alpha = alpha;
    a.kind = kind;
    a.cycles = cycles;
    a.cg_iters = cg_iters;
    a.u0 = u0;
    a.u = u_out;
    a.trace_host = trace_host;
    return run_recon(ctx, a, levels, o, stream, "cm_recon");
}

int cm_fft2d(cm_ctx* ctx, const float* in, float* out, int H, int W, int inverse,
             void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    if (!in || !out || !dims_ok(H, W) || !cm::fft_length_ok(H) || !cm::fft_length_ok(W) ||
        (inverse != 0 && inverse != 1))
        return fail(ctx, CM_ERR_INVALID, "cm_fft2d: invalid argument");
    CM_CUDA(cudaSetDevice(ctx->device));
    cm::FftPlan plan;
    const int rc = cm::fft_plan_make(&plan, H, W);
    if (rc) return fail(ctx, rc == 3 ? CM_ERR_OOM : CM_ERR_CUDA, "cm_fft2d: transform tables");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (out != in)
        e = cudaMemcpyAsync(out, in, (size_t)H * W * 2 * sizeof(float), cudaMemcpyDeviceToDevice,
                            st);
    if (e == cudaSuccess) e = cm::fft2d(plan, reinterpret_cast<float2*>(out), inverse != 0, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cm::fft_plan_free(&plan);
    if (e != cudaSuccess) return fail(ctx, CM_ERR_CUDA, std::string("cm_fft2d: ") + cudaGetErrorString(e));
    return CM_OK;
}

int cm_radon_bins(int H, int W) { return dims_ok(H, W) ? cm::radon_bins(H, W) : -1; }

long long cm_radon_entries(int H, int W, int n_angles) {
    if (!dims_ok(H, W) || n_angles < 1 || n_angles > 100000) return -1;
    const long long m = (long long)n_angles * cm::radon_bins(H, W);
    return m <= CM_MAX_SINO ? m : -1;
}

int cm_radon(cm_ctx* ctx, const float* u, int H, int W, int n_angles, float* sino,
             void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    if (!u || !sino || cm_radon_entries(H, W, n_angles) < 0)
        return fail(ctx, CM_ERR_INVALID, "cm_radon: invalid argument");
    CM_CUDA(cudaSetDevice(ctx->device));
    const char* msg = "";
    const int rc = cm::radon_forward(u, H, W, n_angles, sino, (cudaStream_t)stream, &msg);
    if (rc) return fail(ctx, rc == 3 ? CM_ERR_OOM : CM_ERR_CUDA, std::string("cm_radon: ") + msg);
    return CM_OK;
}

int cm_radon_adjoint(cm_ctx* ctx, const float* sino, int n_angles, int H, int W, float* u,
                     void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    if (!u || !sino || cm_radon_entries(H, W, n_angles) < 0)
        return fail(ctx, CM_ERR_INVALID, "cm_radon_adjoint: invalid argument");
    CM_CUDA(cudaSetDevice(ctx->device));
    const char* msg = "";
    const int rc = cm::radon_adjoint(sino, n_angles, H, W, u, (cudaStream_t)stream, &msg);
    if (rc)
        return fail(ctx, rc == 3 ? CM_ERR_OOM : CM_ERR_CUDA, std::string("cm_radon_adjoint: ") + msg);
    return CM_OK;
}

int cm_recon_ct(cm_ctx* ctx, const float* sino, int n_angles, int H, int W, float alpha,
                int kind, int levels, int cycles, int cg_iters, const float* u0, float* u_out,
                const cm_options* opts, double* trace_host, void* stream) {
    if (!ctx) return CM_ERR_INVALID;
    cm_options o;
    cm_options_default(&o);
    if (opts) o = *opts;
    int rc = check_opts(ctx, o);
    if (rc) return rc;
    if (!sino || !u_out || cm_radon_entries(H, W, n_angles) < 0 || !finite_positive(alpha) ||
        !valid_kind(kind) || levels < 0 || cycles < 0 || cycles > 100000 || cg_iters < 1 ||
        cg_iters > 1000 ||
        (const void*)u_out == (const void*)sino)
        return fail(ctx, CM_ERR_INVALID, "cm_recon_ct: invalid argument");
    cm::ReconArgs a;
    a.op = cm::RECON_CT;
    a.kspace = nullptr;
    a.mask = nullptr;
    a.sino = sino;
    a.n_angles = n_angles;
    a.H = H;
    a.W = W;
    a.alpha = alpha;
    a.kind = kind;
    a.cycles = cycles;
    a.cg_iters = cg_iters;
    a.u0 = u0;
    a.u = u_out;
    a.trace_host = trace_host;
    return run_recon(ctx, a, levels, o, stream, "cm_recon_ct");
}

}  // extern "C"
