/*
 * cm.h -- C ABI of the GB300 multigrid curvature-energy library (libcm.so).
 *
 * The library minimises the discrete curvature energies of "Fast Multi-grid
 * Methods for Minimizing Curvature Energies" (Zhang, Chen, Tang, Duan):
 *
 *   F(u) = sum_pixels |kappa(u)| + alpha/2 (u - f)^2                (Eq. MCM, Eq. GCM)
 *
 * with kappa the mean curvature H = (kmin + kmax)/2 (kind 0) or the Gaussian
 * curvature K = kmin * kmax (kind 1) of the image surface (x, y, u(x, y)),
 * estimated from the eight tangent planes of each 3x3 window (Sec. 2.1,
 * Eq. distance to tri; Sec. 3): kmin and kmax are the extreme curvatures of
 * the four directions W-E, N-S, NW-SE and NE-SW.  Kinds 2 and 3 (an
 * extension, not in the paper) take H and K from a least-squares fit of
 * Euler's formula kappa(theta) = a + b cos 2theta + s sin 2theta to those
 * four direction curvatures instead: principal curvatures a -+ sqrt(b^2 +
 * s^2), H = a (kind 2), K = a^2 - b^2 - s^2 (kind 3), exact in the limit for
 * principal axes at any angle to the pixel grid.  Every entry point that
 * takes `kind` accepts 0..3.  Minimisation is the coloured
 * block-subspace correction sweep: on each level of the fine-to-coarse
 * hierarchy (block sides 1, 2, 4, ...; Sec. 2.2), the blocks of one colour
 * (Sec. 2.3) each find the constant shift c that minimises F(u + c phi_A)
 * and apply it (Alg. 3); cycles repeat until the relative energy change
 * falls to the tolerance (Eq. reerr).
 *
 * Conventions shared by every entry point:
 *  - Images are row-major float32 arrays with row pitch W, H rows.  Unless a
 *    parameter says "host", a pointer is a DEVICE pointer on the context's
 *    device, allocated and owned by the caller; the library never frees it.
 *  - `stream` is a cudaStream_t (0 = the legacy default stream) passed as
 *    void*.  All device work is enqueued on it.  Calls that return a host
 *    value (an energy, statistics) synchronise that stream before returning.
 *  - The library owns only its scratch memory, held by the context and
 *    reused across calls; a context is not safe for concurrent use from
 *    several host threads.
 *  - Every function returns a status code; no exception crosses the ABI.
 *    cm_last_error() gives a message for the last failure on a context.
 *  - Boundary condition: pixels outside the image take the value of the
 *    nearest in-image pixel (clamp to edge).
 */
#ifndef CM_H
#define CM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define CM_OK 0
#define CM_ERR_INVALID 1     /* null pointer, size out of range, alpha <= 0 or non-finite, bad kind/option */
#define CM_ERR_CUDA 2        /* a CUDA runtime call failed (message in cm_last_error) */
#define CM_ERR_OOM 3         /* scratch allocation failed */
#define CM_ERR_TIMEOUT 4     /* a device-side wait hit its iteration limit */
#define CM_ERR_NUMERIC 5     /* NaN or Inf energy */
#define CM_NOT_CONVERGED 6   /* cycle cap reached with tol > 0; u_out is still valid */

/* Image sizes: 1 .. CM_MAX_SIDE rows and columns and at most CM_MAX_PIXELS
 * pixels per image (8 GiB of FP32; block and tile counts are int).  Larger
 * images are rejected with CM_ERR_INVALID (cm_radon_bins returns -1).
 * CM_MAX_SIDE = 65535 x 8: the kernels with the shortest row tiles (8 rows)
 * put the row-tile count in a grid's y dimension, whose limit is 65535. */
#define CM_MAX_SIDE 524280
#define CM_MAX_PIXELS 2147483647LL

#define CM_KIND_MEAN 0
#define CM_KIND_GAUSS 1
#define CM_KIND_MEAN_EULER 2    /* extension: H from the Euler fit */
#define CM_KIND_GAUSS_EULER 3   /* extension: K from the Euler fit */

typedef struct cm_ctx cm_ctx;

/* Solver options.  Fill with cm_options_default() and override fields. */
typedef struct {
    int ncolors;         /* 2: checkerboard of blocks; 4: the paper's four colours (Sec. 2.3);
                            9, 16: 3 x 3, 4 x 4 colours (p (bi mod p) + (bj mod p));
                            0: decoupled, per level the smallest p >= 2 with (p - 1) b >= 3,
                            so that blocks of one colour share no stencil and each colour's
                            parallel solve equals solving its blocks one at a time */
    int grid_points;     /* G: odd, >= 3; points of the bracket grid of the block search */
    int golden_evals;    /* K: >= 2; golden-section evaluations of the block search */
    int paper_candidate; /* 1: also try the paper's one-step FBS estimate on the finest level */
    int use_graph;       /* 1: cm_solve runs as one CUDA graph (device loop and
                            stopping test); 0: one cycle per launch sequence,
                            host stopping test (same results) */
    int max_trace;       /* entries of the energy trace kept in cm_stats (<= 4096) */
    int one_step;        /* 1: instead of the search, every block takes one step of
                            Alg. 2 (t = 0, c_0 = 0, eta = 1): c_1 = (c_1/2 + alpha f*) /
                            (2 + alpha), f* the block mean of f - u, c_1/2 the plane-
                            distance estimate (Eq. c-sol1; Prop. 2 for kind 1) on the
                            finest level and 0 on coarser ones; c_1 is kept if it lowers
                            E_A, else the block keeps 0 (two evaluations per block) */
    int vcycle;          /* 1: full V-cycle, levels 1 .. L then L-1 .. 1 (Sec. 2.2, compared
                            with the half cycle in Sec. 4.1); 0: the half V-cycle of Alg. 3,
                            levels 1 .. L */
    int coarse_spec;     /* coarse levels (b >= 64): -1 the level's default, 0/1 speculate the
                            first golden pair in the grid's reduction */
    int coarse_dmax;     /* coarse levels: 0 the level's default, 1 .. 4 golden steps per
                            reduction (2^d - 1 points of every outcome path); both change only
                            how many candidates share a reduction, never which are taken */
    int coarse_ncolors;  /* levels of block side >= 64: 0 the ncolors rule, or 1, 2, 4, 9, 16
                            colours there (fewer colours: fewer sequential phases on the
                            latency-bound coarse levels; with 2 same-colour blocks share only
                            corner pixels of their rings, with 1 every block of the level
                            solves from the same state in one phase: a block-Jacobi step) */
    int block_sides;     /* 0: block side 2^(j-1) on level j (default); 1: the paper's patches
                            of (2^j - 1) x (2^j - 1) pixels (Sec. 2.2: 1, 3, 7, 15, ...), with
                            levels = 0 meaning the largest side <= min(H, W) / 2.  Levels of
                            odd side run the per-phase kernels (direct block sums and apply) */
    int shapes;          /* kernel shapes of the levels b = 2 .. 32 (power-of-two sides), one
                            bit each, 0 = the default shape (cm_options_default: 0), chosen by
                            the autotuner per shape class; the candidates searched and the
                            tie rule are the same, only the threads per block and the FP32
                            order of the ring sums differ:
                            bit 0 (b = 2):  8 lanes, two ring pixels each, instead of the
                                            rotation-specialised 4-lane kernel;
                            bit 1 (b = 4):  32 lanes, one ring pixel each, instead of 16 x 2;
                            bit 2 (b = 8):  a 64-thread CTA, one ring pixel each, instead of
                                            a warp with two;
                            bit 3 (b = 16): a warp, four ring pixels per lane, instead of a
                                            128-thread CTA with one;
                            bit 4 (b = 32): a 128-thread CTA, two ring pixels per thread,
                                            instead of a 256-thread CTA with one */
} cm_options;

/* Solve statistics (host struct, filled by cm_solve). */
typedef struct {
    int cycles_run;           /* outer iterations performed */
    int converged;            /* 1 if the relative-energy test stopped the loop */
    int monotone_violations;  /* cycles whose energy rose over the previous one */
    int levels;               /* levels used */
    double energy_initial;    /* F(u_0), FP64 device reduction */
    double energy_final;      /* F(u_out) */
    int trace_len;            /* entries written to energy_trace */
    double energy_trace[4097];/* F(u_0), F(u_1), ... (first max_trace + 1 cycles) */
} cm_stats;

/* Default options: ncolors 4 (the paper's four-colour decomposition, Sec. 2.3), G 5, K 6
 * (the budget the autotuner picks on every tested workload: fastest time to tolerance at the
 * lowest final energy), paper_candidate 1, use_graph 1, max_trace 4096, one_step 0,
 * vcycle 0, coarse_spec -1, coarse_dmax 0. */
int cm_options_default(cm_options* opts /* host */);

/* Create a context on CUDA device `device` (makes it current on this
 * thread).  *ctx receives the handle.  Errors: CM_ERR_INVALID (null),
 * CM_ERR_CUDA (no such device). */
int cm_create(cm_ctx** ctx /* host */, int device);

/* Free the context's scratch memory and graphs.  NULL is ignored. */
void cm_destroy(cm_ctx* ctx);

/* Message of the last error on ctx ("" if none).  Valid until the next call. */
const char* cm_last_error(const cm_ctx* ctx);

/* Number of levels used when `levels` = 0: block sides 1, 2, 4, ... up to the
 * largest power of two <= min(H, W)/2 (at least one level). */
int cm_auto_levels(int H, int W);

/* Discrete energy F(u) of Eq. (MCM) (kind 0) or Eq. (GCM) (kind 1).
 * u, f: device, H x W.  Per-pixel terms in FP32, summed in FP32 over each
 * 32 x 32 tile and those sums in FP64, on the device in a fixed order
 * (bit-reproducible).  *E_host (host) receives F.
 * Synchronises `stream`. */
int cm_energy(cm_ctx* ctx, const float* u, const float* f, int H, int W, float alpha,
              int kind, double* E_host, void* stream);

/* Per-pixel curvature kappa (signed H or K) into out (device, H x W). */
int cm_curvature(cm_ctx* ctx, const float* u, int H, int W, int kind, float* out,
                 void* stream);

/* One phase of the sweep (Alg. 3 inner step): on the level with block side
 * b (a power of two), every block of colour `colour` finds the shift
 * c = argmin_c F(u + c phi_A) with the block search below and writes
 * R = u + c on its pixels.  The phase state u is R on blocks of colours <
 * `colour` of this level and S elsewhere (pass S == R-content copies for a
 * plain state).  Blocks of other colours are not written.  All blocks of the
 * colour read the state at the start of the phase.
 * Block search: c_fid = -S1/s (S1 = sum over the block of u - f, s its pixel
 * count); bracket rho = sqrt(2 sum_ring|kappa(c_fid)| / (alpha s)); E_A at
 * G equispaced points of [c_fid - rho, c_fid + rho]; K golden-section
 * evaluations on [g* - D, g* + D] around the best grid point g* (D the grid
 * step); also c = 0 and, for b = 1, the paper's estimate (Eq. c-sol1/c-sol2
 * with t = 0, or Prop. 2 for kind 1); the best evaluated c wins.
 * S, R, f: device H x W; R must not alias S or f.  c_out (device, nullable):
 * receives c for every block of the colour, indexed bi * nbj + bj with
 * nbj = ceil(W / b) (other entries untouched). */
int cm_phase(cm_ctx* ctx, const float* S, float* R, const float* f, int H, int W, float alpha,
             int kind, int b, int colour, const cm_options* opts /* host, nullable */,
             float* c_out, void* stream);

/* One whole level of the sweep (the inner loop of Alg. 3 over the colours
 * k = 0 .. ncolors-1 on the level with block side b, a power of two): from
 * the state S, each colour's blocks in turn find their shift from the state
 * left by the previous colours, exactly as a sequence of cm_phase calls
 * would; R (every pixel) receives the state after the last colour.  This is
 * the path cm_solve runs: on levels with b >= 64 it evaluates block sums from
 * 32 x 32 tile sums and applies all shifts in one pass after the last colour,
 * which changes only the FP32 summation order of S1.
 * S, R, f: device H x W; R must not alias S or f.  c_out (device, nullable):
 * receives every block's c, indexed bi * nbj + bj, nbj = ceil(W / b). */
int cm_level(cm_ctx* ctx, const float* S, float* R, const float* f, int H, int W, float alpha,
             int kind, int b, const cm_options* opts /* host, nullable */, float* c_out,
             void* stream);

/* Full solve (Alg. 3, half V-cycle): u_0 = u0 (or f when u0 is NULL); each
 * cycle sweeps levels 1..L fine to coarse, colours in ascending order; the
 * FP64 energy is evaluated after every cycle and the loop stops when
 * |F_l - F_{l-1}| <= tol |F_l| (Eq. reerr, tol > 0) or after `cycles`
 * cycles (exactly `cycles` when tol == 0).  levels = 0 selects
 * cm_auto_levels(H, W).  f, u0, u_out: device H x W; u_out may alias u0 but
 * not f.  stats (host, nullable).  Returns CM_NOT_CONVERGED if tol > 0 and the
 * cap was reached (u_out valid).  Synchronises `stream`.
 * With use_graph the loop runs on the device: the solve is one CUDA graph
 * (cached per configuration) whose conditional WHILE node repeats a cycle and
 * a one-thread stopping-test kernel that sets the loop condition; the host
 * reads the state back once.  Without it the host tests after every cycle;
 * both give identical u, statistics and energy trace. */
int cm_solve(cm_ctx* ctx, const float* f, int H, int W, float alpha, int kind, int levels,
             int cycles, double tol, const float* u0, float* u_out,
             const cm_options* opts /* host, nullable */, cm_stats* stats /* host, nullable */,
             void* stream);

/* Batched solve: n independent images of uneven sizes (Alg. 3 on each).
 * Arrays f, H, W, alpha, kind, u0 (nullable; entries may be NULL) and u_out
 * are HOST arrays of length n; the image pointers they hold are device
 * pointers.  levels, cycles, tol and opts apply to every image (levels = 0:
 * cm_auto_levels per image).  One CUDA graph holds one cycle of every image
 * (an independent chain per image, so images run concurrently); each image
 * stops on its own relative-energy test (Eq. reerr), evaluated on the device,
 * after which its kernels return at entry.  The cycle sits in the body of a
 * conditional WHILE node whose condition a kernel sets to "some image is
 * active", so the whole batch is one graph launch and one read-back of a
 * small state array (the loop ends: every image stops at `cycles`).  Every
 * image's result and statistics equal those of cm_solve on that image alone
 * (same kernels, same order).  stats: host array of n (nullable).  Returns
 * CM_NOT_CONVERGED if tol > 0 and an image hit the cap, CM_ERR_NUMERIC on a
 * non-finite energy.  Scratch: one context arena (an image-sized buffer and
 * small sums per image).  Synchronises `stream`. */
int cm_solve_batched(cm_ctx* ctx, int n, const float* const* f, const int* H, const int* W,
                     const float* alpha, const int* kind, int levels, int cycles, double tol,
                     const float* const* u0, float* const* u_out,
                     const cm_options* opts /* host, nullable */,
                     cm_stats* stats /* host, n entries, nullable */, void* stream);

/* ---------------------------------------------------------------------------
 * Learned warm start (not in the paper): a small CNN maps f to an initial
 * u0 for the sweep, which then runs from u0 and is both the fallback and the
 * arbiter of the network's output.  Network: six 3x3 convolutions with zero
 * padding, channels 1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU after the first
 * five, residual output u0 = f + conv6(...).  BF16 weights and activations,
 * FP32 accumulation (the 32 -> 32 layers on the tensor cores).
 * Parameters: one flat FP32 vector of cm_net_num_params() = 37601 values:
 * W1 [9][32] (tap, out), b1 [32]; W2..W5 [9][32][32] (tap, in, out),
 * b2..b5 [32]; W6 [9][32] (tap, in), b6 [1]; tap = (dy + 1) * 3 + (dx + 1). */
typedef struct cm_net cm_net;

int cm_net_num_params(void);
/* Create a network on the current device with all parameters zero (then
 * u0 = f).  ctx is only checked for validity. */
int cm_net_create(cm_ctx* ctx, cm_net** net /* host */);
void cm_net_destroy(cm_net* net);
const char* cm_net_last_error(const cm_net* net);
/* Host FP32 parameter vector in / out; setting resets the Adam moments. */
int cm_net_set_params(cm_net* net, const float* params_host);
int cm_net_get_params(cm_net* net, float* params_host);
/* u0 = f + net(f): f, u0_out device, N images of H x W, row-major.  Every
 * cm_net_* call on images takes N H W < 2^31 (else CM_ERR_INVALID). */
int cm_net_forward(cm_net* net, const float* f, int N, int H, int W, float* u0_out, void* stream);
/* Gradient of the loss mean((u0 - u*)^2) over all N H W pixels (grad_host:
 * 37601 floats, nullable; loss_host nullable).  Synchronises `stream`. */
int cm_net_gradients(cm_net* net, const float* f, const float* ustar, int N, int H, int W,
                     float* grad_host, double* loss_host, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on that
 * loss for the batch (f, u*), device pointers.  loss_host (nullable) receives
 * the loss before the step (synchronising `stream`). */
int cm_net_train_step(cm_net* net, const float* f, const float* ustar, int N, int H, int W,
                      float lr, double* loss_host, void* stream);
/* Checkpoint of a network: the FP32 parameters, the Adam moments and the
 * Adam step count, so that training resumes exactly.  File layout
 * (little-endian): "CMNETCK1", uint32 version 1, uint32 parameter count
 * (37601), uint64 step; float params[n], m[n], v[n]; uint32 CRC-32 (IEEE
 * 802.3) of all preceding bytes.  cm_net_load rejects a file of another
 * size, header or checksum with CM_ERR_INVALID (the network is unchanged);
 * an unopenable path is CM_ERR_INVALID too (message in cm_net_last_error).
 * Both synchronise the device. */
int cm_net_save(cm_net* net, const char* path);
int cm_net_load(cm_net* net, const char* path);

/* Training loop (mean((u0 - u*)^2), Adam as in cm_net_train_step). */
typedef struct {
    int steps;          /* Adam steps of this call (>= 1) */
    int batch;          /* pairs per step, 1 .. N, drawn without replacement */
    float lr;           /* learning rate at schedule step 0 (> 0) ... */
    float lr_final;     /* ... decaying by a cosine to this at step total_steps - 1 (> 0) */
    int total_steps;    /* schedule length; 0: start_step + steps */
    int start_step;     /* schedule index of this call's first step (resume after a checkpoint) */
    uint64_t seed;      /* mini-batch sampling */
    int log_every;      /* record the loss of every log_every-th step of the call (>= 1) */
} cm_train_opts;

typedef struct {
    double loss_first;  /* loss of the call's first step, before its update */
    double loss_last;   /* loss of the call's last step, before its update */
    int n_logged;       /* entries written */
    int losses_cap;     /* capacity of the arrays below */
    double* losses;     /* host, losses_cap entries (nullable when losses_cap = 0) */
    int* logged_steps;  /* host, nullable: schedule index of each logged loss */
} cm_train_log;

/* Trains `net` on N device pairs f[i], ustar[i] (each H x W, row-major,
 * consecutive).  Step t (t = start_step .. start_step + steps - 1) uses the
 * pairs of a partial Fisher-Yates shuffle of 0 .. N-1 driven by SplitMix64:
 * the stream's state is its (t + 1)-th output from `seed`, draw j its
 * (j + 1)-th output from that state, and r = j + draw mod (N - j) is swapped
 * into place j; the pairs are copied into a scratch batch and one Adam step
 * runs with lr_t = lr_final + (lr - lr_final)(1 + cos(pi t / max(1, T - 1)))/2,
 * T = total_steps.  Calls with consecutive step ranges of one schedule, with
 * a checkpoint in between, give the same parameters as one call.  log
 * (host, nullable) receives the losses.  Synchronises `stream`. */
int cm_net_train(cm_ctx* ctx, cm_net* net, const float* f, const float* ustar, int N, int H,
                 int W, const cm_train_opts* opts, cm_train_log* log, void* stream);

/* u0_out = f + net(f) for N images; with check_energy, an image keeps u0
 * only if F(u0) <= F(f) (energies of Eq. MCM/GCM with alpha and kind), else
 * u0 = f.  used_host (nullable, N ints) receives 1 where u0 was kept. */
int cm_warmstart(cm_ctx* ctx, cm_net* net, const float* f, int N, int H, int W, float* u0_out,
                 int check_energy, float alpha, int kind, int* used_host, void* stream);

/* Energy without allocation.  The paper has no counterpart: this is a
 * service for callers that cannot let a library allocate device memory -- a
 * host whose caching allocator already holds (nearly) all of it, code that
 * must not take the implicit device-wide synchronisation of cudaMalloc and
 * cudaFree, or a pipeline that forbids allocation after start-up.  It
 * computes the same F(u) as cm_energy with the same kernel, but takes no
 * context and allocates nothing: its scratch (one FP64 partial per 32 x 32
 * tile and an arrival counter) is a fixed array inside the library, about
 * 128 KiB, which every GPU that loads the library holds until the process
 * exits.
 * u, f: device, H x W, row-major float32 on the current device.  E_dev:
 * device pointer to one double that receives F(u) when the work on `stream`
 * completes (the call does not synchronise).
 * Returns CM_ERR_INVALID for null pointers, sizes < 1 or beyond CM_MAX_SIDE
 * and CM_MAX_PIXELS, a bad alpha or kind,
 * and for images with more than CM_NOALLOC_MAX_TILES tiles of 32 x 32 pixels
 * (ceil(H/32) * ceil(W/32) > 16384, e.g. larger than 4096 x 4096);
 * CM_ERR_CUDA if a CUDA call fails.
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it until the process exits; make that first call
 * before any stream capture, and make no call on a device after
 * cudaDeviceReset of it (the kept address is then stale).  Every
 * call shares the one array and clears its counter before use, so calls whose
 * work overlaps on the GPU (on different streams, or from several host
 * threads without ordering) race and must be serialised by the caller. */
#define CM_NOALLOC_MAX_TILES 16384
int cm_energy_noalloc(const float* u, const float* f, int H, int W, float alpha, int kind,
                      double* E_dev, void* stream);

/* Reconstruction extension (Sec. 5), MRI-like operator: recovers a real
 * H x W image u from k-space data b by minimising
 *     J(u) = 1/2 ||A u - b||^2 + alpha sum |kappa(u)|,
 * A = M F with F the orthonormal 2-D DFT (unitary: F^H F = I, the DC entry is
 * sum(u) / sqrt(HW)) and M the 0/1 mask of sampled entries.  Each cycle
 * visits the levels fine to coarse and the colours in order (Alg. 3); the
 * blocks phi_i of one colour are corrected together by cg_iters conjugate-
 * gradient iterations (from c = 0; stopping early only on a zero residual or
 * a non-positive p.Ap) on the normal equations of Sec. 5,
 *     [Re<A phi_i, A phi_j> + 2 alpha delta_ij] c = Re<b - A u, A phi_i> + 2 alpha d_i,
 * with d_i = c_{1/2} of Eq. c-sol1 (Prop. 2 for kinds 1 and 3) on the finest
 * level and 0 on coarser ones.
 * kspace: device, H x W complex values as (re, im) float pairs, row-major,
 * zero off the mask.  mask: device, H x W bytes, 0 or 1.  u0: device H x W or
 * NULL (start from the zero-filled Re(A^H b)); u_out: device H x W (may
 * alias u0).  levels = 0: cm_auto_levels rule (opts->block_sides applies, as
 * do opts->ncolors; the search options do not).  trace_host (nullable, host,
 * cycles + 1 doubles) receives J before the first cycle and after each.
 * The transforms are the library's own (cm_fft2d below), so H and W are
 * each a power of two up to CM_FFT_MAX_POW2 or any length up to
 * CM_FFT_MAX_OTHER; the scratch (two complex images, the transform tables and
 * the CG vectors) stays in the context.  Synchronises `stream`.  Returns
 * CM_ERR_INVALID for null pointers, sizes out of range (CM_MAX_SIDE,
 * CM_MAX_PIXELS, the transform's limits), u_out aliasing kspace, a bad alpha,
 * kind or option, cycles outside 0 .. 100000 or cg_iters outside 1 .. 1000;
 * CM_ERR_OOM when the scratch cannot be allocated; CM_ERR_CUDA otherwise on a
 * failed CUDA call. */
/* The 2-D discrete Fourier transform of the MRI-like operator A = M F
 * (Sec. 5), unnormalised: out[k, l] = sum_{r, c} in[r, c]
 * exp(-+2 pi i (k r / H + l c / W)) with the minus sign (inverse = 0) or the
 * plus sign (inverse = 1); the orthonormal F is this times 1/sqrt(HW).  in,
 * out: device, H x W complex values as (re, im) float pairs, row-major; out
 * may equal in (in place).  FP32 arithmetic with twiddle and chirp tables
 * computed in FP64: rows, then columns, each line in one CTA's shared memory
 * (radix-2; a length that is not a power of two by Bluestein's chirp
 * z-transform with a power-of-two length >= 2n - 1).  Allocates the tables
 * for the call and frees them; synchronises `stream`.  Returns CM_ERR_INVALID
 * for null pointers, inverse not 0 or 1, and sizes other than a power of two
 * <= CM_FFT_MAX_POW2 or a length <= CM_FFT_MAX_OTHER per axis; CM_ERR_OOM or
 * CM_ERR_CUDA on a failed allocation or CUDA call. */
#define CM_FFT_MAX_POW2 16384
#define CM_FFT_MAX_OTHER 8192
int cm_fft2d(cm_ctx* ctx, const float* in, float* out, int H, int W, int inverse, void* stream);

int cm_recon(cm_ctx* ctx, const float* kspace, const unsigned char* mask, int H, int W,
             float alpha, int kind, int levels, int cycles, int cg_iters, const float* u0,
             float* u_out, const cm_options* opts /* host, nullable */,
             double* trace_host /* host, nullable */, void* stream);

/* Reconstruction extension, CT case (Sec. 5 with A = R, a parallel-beam
 * Radon transform): the same sweep and per-colour conjugate gradients as
 * cm_recon, with the normal equations of R.  Geometry (a reading: Sec. 5
 * names the Radon transform but no discretisation): n_angles angles
 * theta_a = pi a / n_angles; the centre of pixel (r, c) is at
 * x = c - (W-1)/2, y = r - (H-1)/2 and projects to p = x cos theta + y sin
 * theta + (D-1)/2 on a detector of D = cm_radon_bins(H, W) =
 * 2 ceil(hypot(H-1, W-1)/2) + 3 unit bins; the pixel's value goes to bins
 * floor(p) and floor(p) + 1 with weights 1 - frac(p), frac(p) (every p lies
 * in [1, D-2]).  sino: device, n_angles x D row-major float32.  u0: device
 * H x W or NULL: start from the filtered backprojection (pi / n_angles)
 * R^T (h * b), h the Ram-Lak kernel (h[0] = 1/4, h[k] = -1/(pi k)^2 for odd k,
 * 0 for even k, a direct convolution per angle).  trace_host as in
 * cm_recon; the CG and colour options as in cm_recon; no Fourier transform.
 * Synchronises `stream`.  Returns CM_ERR_INVALID for null pointers, sizes out
 * of range, n_angles outside 1 .. 100000, u_out aliasing sino, a bad alpha,
 * kind or option, cycles outside 0 .. 100000 or cg_iters outside 1 .. 1000;
 * CM_ERR_OOM or CM_ERR_CUDA as cm_recon.  The sinogram is indexed with
 * int: n_angles x D above CM_MAX_SINO entries is rejected with
 * CM_ERR_INVALID by every CT entry point.  cm_radon_bins and
 * cm_radon_entries are host-only: D, or the sinogram's entry count
 * n_angles x D, or -1 where the image size, n_angles or the entry count is
 * out of range. */
#define CM_MAX_SINO 2147483647LL
int cm_radon_bins(int H, int W);
long long cm_radon_entries(int H, int W, int n_angles);
int cm_recon_ct(cm_ctx* ctx, const float* sino, int n_angles, int H, int W, float alpha,
                int kind, int levels, int cycles, int cg_iters, const float* u0, float* u_out,
                const cm_options* opts /* host, nullable */,
                double* trace_host /* host, nullable */, void* stream);
/* The CT operator pair alone: sino = R u (n_angles x D), u = R^T sino (the
 * exact transpose: both are gathers with the same weights).  Device
 * pointers, caller-owned: u is H x W and sino n_angles x D, both row-major
 * float32; temporaries are allocated and freed; synchronise `stream`.
 * Return CM_ERR_INVALID for null pointers, sizes out of range or n_angles
 * outside 1 .. 100000, CM_ERR_OOM, or CM_ERR_CUDA. */
int cm_radon(cm_ctx* ctx, const float* u, int H, int W, int n_angles, float* sino,
             void* stream);
int cm_radon_adjoint(cm_ctx* ctx, const float* sino, int n_angles, int H, int W, float* u,
                     void* stream);

/* Measurement support (not part of the solver).  The sweep kernels are bound
 * by FP32 and MUFU instruction issue, so their roofline is taken against the
 * GPU's measured arithmetic rates: fma_per_s (host) receives FP32 fused
 * multiply-adds per second, rsqrt_per_s (host) rsqrtf operations per second
 * (one MUFU instruction each), each from a fixed-work kernel of eight
 * independent dependency chains per thread on every SM (8 CTAs of 256
 * threads per SM), timed with CUDA events on `stream` after a warm-up launch
 * (about 10 ms each at the nominal rates).  Allocates and frees 4 bytes of
 * device memory on `device`; synchronises `stream`.  Returns CM_ERR_INVALID
 * for null pointers or a negative device, CM_ERR_OOM, or CM_ERR_CUDA. */
int cm_probe_alu(int device, double* fma_per_s, double* rsqrt_per_s, void* stream);

/* Failure detection.  Every wait of the library's kernels on an mbarrier (the
 * tensor-core convolution's pipeline) gives up after a bounded number of
 * tries, sets an error status and returns; the entry points that synchronise
 * report it as CM_ERR_TIMEOUT, and the context stays usable.  This self-test
 * runs that wait in one CTA on phase 0 of a fresh mbarrier (arrival count 1)
 * that nothing completes, with `limit` tries (1 .. 2^22): *timed_out = 1 when
 * the wait gave up; it then arrives once and waits again: *completed = 1 when
 * that wait saw the phase complete.  Host pointers; synchronises the device.
 * Out-of-memory is injected on the host: with CM_FAULT_ALLOC_LIMIT=<bytes> in
 * the environment, a context's scratch allocations larger than that fail as
 * CM_ERR_OOM. */
int cm_selftest_wait(int device, int limit, int* timed_out, int* completed);

#ifdef __cplusplus
}
#endif

#endif /* CM_H */
