// cm_fft.cu -- 2-D DFT of the MRI-like operator A = M F (Sec. 5).
//
// The 2-D transform is a pass of 1-D transforms along the rows followed by
// a pass along the columns.  One CTA transforms L whole lines in shared
// memory with radix-4 stages (radix-2 for an odd stage count), one CTA
// barrier per stage: up to 8192 points per CTA in the self-sorting
// (Stockham) form, two padded copies in natural order; longer lines in
// place, loaded in bit-reversed order, as decimation-in-time stages taken
// two at a time in registers.  A column pass loads L >= 4 neighbouring columns at once, so
// every row segment it reads or writes is L consecutive complex values.
//
// Lines whose length n is not a power of two use Bluestein's chirp
// z-transform: with jk = (j^2 + k^2 - (k - j)^2) / 2,
//   X_k = w_k sum_j (x_j w_j) conj(w_{k-j}),   w_m = exp(-i pi m^2 / n)
// (forward; the inverse conjugates every w), a convolution evaluated with
// transforms of a power of two M >= 2n - 1: the chirped line is transformed,
// multiplied by the precomputed spectrum of the chirp (divided by M) and
// transformed back, then chirped again.
//
// Twiddles exp(-2 pi i m / M), the chirps and the chirp spectra are computed
// in FP64 on the host (the spectrum with a host FFT of its own) and stored as
// FP32 tables; the arithmetic on the device is FP32.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "../../include/cm.h"
#include "cm_fft.h"

namespace cm {

static_assert(CM_FFT_MAX_POW2 == FFT_MAX_M && CM_FFT_MAX_OTHER == FFT_MAX_M / 2,
              "transform limits of include/cm.h");

constexpr int FFT_THREADS = 256;
// Lines per CTA: about 1024 points (two radix-4 groups per thread and step),
// at least four columns in a column pass (32-byte row segments), at most
// 8192 points (64 KB of shared memory) unless one line is longer.
constexpr int FFT_TARGET_POINTS = 1024;
constexpr int FFT_POINTS_PER_CTA = 8192;
constexpr int FFT_MIN_COLS = 4;
// The self-sorting kernel holds two padded copies of its lines: up to 8192
// points per CTA (2 x 9216 x 8 bytes of shared memory); longer lines use the
// in-place kernel.
constexpr int FFT_STOCK_POINTS = 8192;
constexpr int FFT_STOCK_SMEM = 2 * (FFT_STOCK_POINTS + FFT_STOCK_POINTS / 8 + 64) * 8;
// Line pitch in the self-sorting kernel's shared memory: spad(M) + 4 float2,
// so that the L lines of a column pass, read and written a row at a time,
// start in different banks.
__host__ __device__ __forceinline__ int stock_pitch(int M) { return M + (M >> 3) + 4; }

struct FftAxis {
    int n = 0, M = 0, log2M = 0;
    int L = 1;        // lines per CTA of a row pass
    int Lc = 1;       // lines per CTA of a column pass
    bool pow2 = true;
    float2* tw = nullptr;      // M / 2: exp(-2 pi i m / M)
    float2* chirp = nullptr;   // n: exp(-i pi k^2 / n) (Bluestein only)
    float2* Bf = nullptr;      // M: spectrum of the forward chirp kernel / M
    float2* Bi = nullptr;      // M: spectrum of the inverse chirp kernel / M
};

bool fft_length_ok(int n) {
    if (n < 1) return false;
    if ((n & (n - 1)) == 0) return n <= FFT_MAX_M;
    return n <= FFT_MAX_M / 2;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// log2M decimation-in-time stages over L lines of M points held in
// bit-reversed order in P (line l at P + l * M); twiddles conjugated for the
// inverse.  Stages s and s + 1 run as one radix-4 step: the four points a0,
// a0 + h, a0 + 2h, a0 + 3h (h = 2^(s-1)) take the two radix-2 butterflies of
// stage s (twiddle of index k for span 2^s) and then those of stage s + 1
// (indices k and k + h for span 2^(s+1)) in registers, so each pair of
// stages costs one pass through shared memory and one barrier; an odd stage
// count ends with one radix-2 stage.
__device__ void fft_stages(float2* P, int M, int log2M, int L, const float2* __restrict__ tw,
                           bool inverse) {
    int s = 1;
    for (; s + 1 <= log2M; s += 2) {
        const int half = 1 << (s - 1);
        const int quarter_total = L * (M >> 2);
        for (int t = threadIdx.x; t < quarter_total; t += blockDim.x) {
            const int l = t >> (log2M - 2);
            const int j = t & ((M >> 2) - 1);
            const int k = j & (half - 1);
            const int a0 = l * M + ((j >> (s - 1)) << (s + 1)) + k;
            float2 wA = tw[k * (M >> s)];
            float2 wB0 = tw[k * (M >> (s + 1))];
            float2 wB1 = tw[(k + half) * (M >> (s + 1))];
            if (inverse) {
                wA = conjf2(wA);
                wB0 = conjf2(wB0);
                wB1 = conjf2(wB1);
            }
            const float2 x0 = P[a0];
            const float2 x1 = cmul(P[a0 + half], wA);
            const float2 x2 = P[a0 + 2 * half];
            const float2 x3 = cmul(P[a0 + 3 * half], wA);
            const float2 y0 = make_float2(x0.x + x1.x, x0.y + x1.y);
            const float2 y1 = make_float2(x0.x - x1.x, x0.y - x1.y);
            const float2 z2 = cmul(make_float2(x2.x + x3.x, x2.y + x3.y), wB0);
            const float2 z3 = cmul(make_float2(x2.x - x3.x, x2.y - x3.y), wB1);
            P[a0] = make_float2(y0.x + z2.x, y0.y + z2.y);
            P[a0 + 2 * half] = make_float2(y0.x - z2.x, y0.y - z2.y);
            P[a0 + half] = make_float2(y1.x + z3.x, y1.y + z3.y);
            P[a0 + 3 * half] = make_float2(y1.x - z3.x, y1.y - z3.y);
        }
        __syncthreads();
    }
    if (s == log2M) {
        const int half = 1 << (s - 1);
        const int tstep = M >> s;   // exp(-2 pi i k / 2^s) = tw[k M / 2^s]
        const int half_total = L * (M >> 1);
        for (int t = threadIdx.x; t < half_total; t += blockDim.x) {
            const int l = t >> (log2M - 1);
            const int j = t & ((M >> 1) - 1);
            const int k = j & (half - 1);
            const int i0 = l * M + ((j >> (s - 1)) << s) + k;
            float2 w = tw[k * tstep];
            if (inverse) w = conjf2(w);
            const float2 a = P[i0];
            const float2 b = cmul(P[i0 + half], w);
            P[i0] = make_float2(a.x + b.x, a.y + b.y);
            P[i0 + half] = make_float2(a.x - b.x, a.y - b.y);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int bitrev(int i, int bits) { return (int)(__brev((unsigned)i) >> (32 - bits)); }

// Self-sorting (Stockham) form, used when two copies of the CTA's lines fit
// in shared memory: the lines stay in natural order and every stage reads
// buffer x and writes buffer y.  A radix-4 stage combines four transforms of
// size Ns into one of size 4 Ns: group j (k = j mod Ns) takes a_t = x[j + t M
// / 4] w^(t k) (w = exp(-+2 pi i / (4 Ns))), a 4-point DFT, and writes b_t to
// y[4 (j - k) + k + t Ns]; an odd stage count ends with the radix-2 stage.
// Reads are unit-stride; shared-memory indices carry one float2 of padding
// per 8 (spad) so that the strided writes of the first stages spread over
// the banks.  (The in-place decimation-in-time form above loads in
// bit-reversed order, 32 consecutive points into one bank.)
__device__ __forceinline__ int spad(int i) { return i + (i >> 3); }

// exp(-2 pi i m / M), conjugated for the inverse, 0 <= m < M, from the half
// table tw (m >= M / 2: minus the entry m - M / 2).
__device__ __forceinline__ float2 twid(const float2* __restrict__ tw, int m, int M, bool inverse) {
    const int h = M >> 1;
    float2 w = m < h ? tw[m] : tw[m - h];
    if (m >= h) w = make_float2(-w.x, -w.y);
    return inverse ? conjf2(w) : w;
}

// The stages over L lines of M points (line l at offset l * Mp in x and y);
// returns the buffer that holds the result.
__device__ float2* fft_stockham(float2* x, float2* y, int M, int log2M, int L, int Mp,
                                const float2* __restrict__ tw, bool inverse) {
    int Ns = 1;
    const int Q = M >> 2;
    for (int st = 0; st + 2 <= log2M; st += 2) {
        const int total = L * Q;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int l = t >> (log2M - 2), j = t & (Q - 1);
            const int k = j & (Ns - 1);
            const float2* xl = x + (size_t)l * Mp;
            float2 a0 = xl[spad(j)], a1 = xl[spad(j + Q)], a2 = xl[spad(j + 2 * Q)],
                   a3 = xl[spad(j + 3 * Q)];
            if (Ns > 1) {
                const int m = k * (M / (4 * Ns));   // exp(-+2 pi i t k / (4 Ns)) = twid(t m)
                a1 = cmul(a1, twid(tw, m, M, inverse));
                a2 = cmul(a2, twid(tw, 2 * m, M, inverse));
                a3 = cmul(a3, twid(tw, 3 * m, M, inverse));
            }
            const float2 s02 = make_float2(a0.x + a2.x, a0.y + a2.y);
            const float2 d02 = make_float2(a0.x - a2.x, a0.y - a2.y);
            const float2 s13 = make_float2(a1.x + a3.x, a1.y + a3.y);
            const float2 d13 = make_float2(a1.x - a3.x, a1.y - a3.y);
            // -i d13 (forward), +i d13 (inverse)
            const float2 r = inverse ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
            const int base = ((j - k) << 2) + k;
            float2* yl = y + (size_t)l * Mp;
            yl[spad(base)] = make_float2(s02.x + s13.x, s02.y + s13.y);
            yl[spad(base + Ns)] = make_float2(d02.x + r.x, d02.y + r.y);
            yl[spad(base + 2 * Ns)] = make_float2(s02.x - s13.x, s02.y - s13.y);
            yl[spad(base + 3 * Ns)] = make_float2(d02.x - r.x, d02.y - r.y);
        }
        __syncthreads();
        float2* tmp = x;
        x = y;
        y = tmp;
        Ns <<= 2;
    }
    if (log2M & 1) {   // Ns = M / 2: k = j
        const int hM = M >> 1;
        const int total = L * hM;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int l = t >> (log2M - 1), j = t & (hM - 1);
            const float2* xl = x + (size_t)l * Mp;
            const float2 a0 = xl[spad(j)];
            float2 a1 = xl[spad(j + hM)];
            if (Ns > 1) a1 = cmul(a1, twid(tw, j, M, inverse));   // exp(-+2 pi i j / M)
            float2* yl = y + (size_t)l * Mp;
            yl[spad(j)] = make_float2(a0.x + a1.x, a0.y + a1.y);
            yl[spad(j + hM)] = make_float2(a0.x - a1.x, a0.y - a1.y);
        }
        __syncthreads();
        x = y;
    }
    return x;
}

// fft_lines_kernel with the self-sorting stages: shared memory holds two
// copies of the L lines (padded); Bluestein's two transforms need no
// reordering in between.  Launched with one thread per radix-4 group of a
// stage (L M / 4, at most 1024), so a column pass of few wide CTAs still
// keeps its SMs busy.
template <bool POW2, bool COLS>
__global__ void __launch_bounds__(1024) fft_lines_stockham_kernel(
    float2* __restrict__ X, int n, int M, int log2M, int L, long long elem_stride,
    long long line_stride, int nlines, const float2* __restrict__ tw,
    const float2* __restrict__ chirp, const float2* __restrict__ B, int inverse,
    const uint8_t* __restrict__ mask, float mscale) {
    extern __shared__ float2 P[];
    const int Mp = stock_pitch(M);
    float2* P0 = P;
    float2* P1 = P + (size_t)L * Mp;
    const int l0 = blockIdx.x * L;
    const int nl = min(L, nlines - l0);
    const bool inv = inverse != 0;
    for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
        const int l = COLS ? t % L : t >> log2M;
        const int e = COLS ? t / L : t & (M - 1);
        float2 v = make_float2(0.0f, 0.0f);
        if (l < nl && e < n) {
            v = X[(size_t)(l0 + l) * line_stride + (size_t)e * elem_stride];
            if (!POW2) v = cmul(v, inv ? conjf2(chirp[e]) : chirp[e]);
        }
        P0[(size_t)l * Mp + spad(e)] = v;
    }
    __syncthreads();
    float2* R = fft_stockham(P0, P1, M, log2M, L, Mp, tw, POW2 ? inv : false);
    if (!POW2) {
        for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
            const int l = t >> log2M, e = t & (M - 1);
            float2* q = R + (size_t)l * Mp + spad(e);
            *q = cmul(*q, B[e]);
        }
        __syncthreads();
        R = fft_stockham(R, R == P0 ? P1 : P0, M, log2M, L, Mp, tw, true);
    }
    for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
        const int l = COLS ? t % L : t >> log2M;
        const int e = COLS ? t / L : t & (M - 1);
        if (l < nl && e < n) {
            float2 v = R[(size_t)l * Mp + spad(e)];
            if (!POW2) v = cmul(v, inv ? conjf2(chirp[e]) : chirp[e]);
            const size_t o = (size_t)(l0 + l) * line_stride + (size_t)e * elem_stride;
            if (mask) v = mask[o] ? make_float2(v.x * mscale, v.y * mscale) : make_float2(0.0f, 0.0f);
            X[o] = v;
        }
    }
}

// Transforms nlines lines of X (element e of line l at X[l * line_stride +
// e * elem_stride]) in place.  COLS: the lines are columns (line_stride 1),
// so consecutive threads take consecutive lines; else consecutive elements.
template <bool POW2, bool COLS>
__global__ void __launch_bounds__(FFT_THREADS) fft_lines_kernel(
    float2* __restrict__ X, int n, int M, int log2M, int L, long long elem_stride,
    long long line_stride, int nlines, const float2* __restrict__ tw,
    const float2* __restrict__ chirp, const float2* __restrict__ B, int inverse,
    const uint8_t* __restrict__ mask, float mscale) {
    extern __shared__ float2 P[];
    const int l0 = blockIdx.x * L;
    const int nl = min(L, nlines - l0);
    const bool inv = inverse != 0;
    for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
        const int l = COLS ? t % L : t >> log2M;
        const int e = COLS ? t / L : t & (M - 1);
        float2 v = make_float2(0.0f, 0.0f);
        if (l < nl && e < n) {
            v = X[(size_t)(l0 + l) * line_stride + (size_t)e * elem_stride];
            if (!POW2) v = cmul(v, inv ? conjf2(chirp[e]) : chirp[e]);
        }
        P[(size_t)l * M + bitrev(e, log2M)] = v;
    }
    __syncthreads();
    // POW2: the transform itself.  Bluestein: the forward transform of the
    // chirped line, the product with the chirp spectrum, the inverse.
    fft_stages(P, M, log2M, L, tw, POW2 ? inv : false);
    if (!POW2) {
        for (int t = threadIdx.x; t < L * M; t += blockDim.x) P[t] = cmul(P[t], B[t & (M - 1)]);
        __syncthreads();
        for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
            const int e = t & (M - 1), r = bitrev(e, log2M);
            if (e < r) {
                float2* line = P + (size_t)(t >> log2M) * M;
                const float2 a = line[e];
                line[e] = line[r];
                line[r] = a;
            }
        }
        __syncthreads();
        fft_stages(P, M, log2M, L, tw, true);
    }
    for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
        const int l = COLS ? t % L : t >> log2M;
        const int e = COLS ? t / L : t & (M - 1);
        if (l < nl && e < n) {
            float2 v = P[(size_t)l * M + e];
            if (!POW2) v = cmul(v, inv ? conjf2(chirp[e]) : chirp[e]);
            const size_t o = (size_t)(l0 + l) * line_stride + (size_t)e * elem_stride;
            if (mask) v = mask[o] ? make_float2(v.x * mscale, v.y * mscale) : make_float2(0.0f, 0.0f);
            X[o] = v;
        }
    }
}



cudaError_t fft_setup() {
    const int bytes = FFT_MAX_M * (int)sizeof(float2);   // L * M <= max(8192, FFT_MAX_M)
    cudaError_t e = cudaFuncSetAttribute(fft_lines_kernel<true, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft_lines_kernel<true, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft_lines_kernel<false, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft_lines_kernel<false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft_lines_stockham_kernel<true, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_STOCK_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft_lines_stockham_kernel<true, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_STOCK_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft_lines_stockham_kernel<false, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_STOCK_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft_lines_stockham_kernel<false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_STOCK_SMEM);
    return e;
}

// ---------------------------------------------------------------------------
// Host: tables.

using cd = std::complex<double>;

// Iterative radix-2 FFT in FP64 (forward sign), n a power of two.
static void host_fft(std::vector<cd>& a) {
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = -2.0 * M_PI / (double)len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const cd w(cos(ang * (double)k), sin(ang * (double)k));
                const cd u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

static int upload(float2** dst, const std::vector<cd>& v) {
    std::vector<float2> h(v.size());
    for (size_t i = 0; i < v.size(); ++i) h[i] = make_float2((float)v[i].real(), (float)v[i].imag());
    cudaError_t e = cudaMalloc(dst, h.size() * sizeof(float2));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? 3 : 2;
    e = cudaMemcpy(*dst, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? 0 : 2;
}

static void axis_free(FftAxis* a) {
    if (!a) return;
    cudaFree(a->tw);
    cudaFree(a->chirp);
    cudaFree(a->Bf);
    cudaFree(a->Bi);
    delete a;
}

static int axis_make(FftAxis** out, int n) {
    if (!fft_length_ok(n)) return 1;
    FftAxis* a = new FftAxis();
    a->n = n;
    a->pow2 = (n & (n - 1)) == 0;
    int M = 1;
    while (M < (a->pow2 ? n : 2 * n - 1)) M <<= 1;
    a->M = M;
    while ((1 << a->log2M) < M) ++a->log2M;
    a->L = std::max(1, FFT_TARGET_POINTS / M);
    a->Lc = std::max(1, std::min(std::max(FFT_MIN_COLS, FFT_TARGET_POINTS / M),
                                 FFT_POINTS_PER_CTA / M));
    std::vector<cd> tw(std::max(1, M / 2));
    for (int m = 0; m < M / 2; ++m) tw[m] = std::polar(1.0, -2.0 * M_PI * m / (double)M);
    int rc = upload(&a->tw, tw);
    if (rc == 0 && !a->pow2) {
        // w_k = exp(-i pi k^2 / n), the phase reduced mod 2n exactly in integers
        std::vector<cd> chirp(n), bf(M, cd(0.0, 0.0)), bi(M, cd(0.0, 0.0));
        for (int k = 0; k < n; ++k) {
            const long long q = ((long long)k * k) % (2LL * n);
            chirp[k] = std::polar(1.0, -M_PI * (double)q / (double)n);
        }
        // convolution kernels conj(w_m) (forward) and w_m (inverse), m = -(n-1) .. n-1
        for (int k = 0; k < n; ++k) {
            bf[k] = std::conj(chirp[k]);
            bi[k] = chirp[k];
            if (k > 0) {
                bf[M - k] = bf[k];
                bi[M - k] = bi[k];
            }
        }
        host_fft(bf);
        host_fft(bi);
        for (int m = 0; m < M; ++m) {
            bf[m] /= (double)M;
            bi[m] /= (double)M;
        }
        rc = upload(&a->chirp, chirp);
        if (rc == 0) rc = upload(&a->Bf, bf);
        if (rc == 0) rc = upload(&a->Bi, bi);
    }
    if (rc != 0) {
        axis_free(a);
        return rc;
    }
    *out = a;
    return 0;
}

int fft_plan_make(FftPlan* p, int H, int W) {
    fft_plan_free(p);
    if (!fft_length_ok(H) || !fft_length_ok(W)) return 1;
    int rc = axis_make(&p->rows, W);
    if (rc == 0) rc = axis_make(&p->cols, H);
    if (rc != 0) {
        fft_plan_free(p);
        return rc;
    }
    p->H = H;
    p->W = W;
    return 0;
}

void fft_plan_free(FftPlan* p) {
    axis_free(p->rows);
    axis_free(p->cols);
    p->rows = p->cols = nullptr;
    p->H = p->W = 0;
}

template <bool COLS>
static cudaError_t lines(const FftAxis& a, float2* X, long long elem_stride, long long line_stride,
                         int nlines, bool inverse, cudaStream_t st, const uint8_t* mask = nullptr,
                         float mscale = 1.0f) {
    const int L = COLS ? a.Lc : a.L;
    const dim3 grid((unsigned)((nlines + L - 1) / L));
    const size_t sm = (size_t)L * a.M * sizeof(float2);
    const float2* B = inverse ? a.Bi : a.Bf;
    // self-sorting kernel: fewer lines per CTA when the pass has few lines,
    // aiming at about 256 CTAs (a column pass keeps two or more columns per
    // CTA, so its row segments stay 16 bytes or longer)
    const int Ls = std::min(L, std::max(COLS ? 2 : 1, nlines / 256));
    const size_t sm2 = 2 * (size_t)Ls * stock_pitch(a.M) * sizeof(float2);
    if ((long long)Ls * a.M <= FFT_STOCK_POINTS && sm2 <= (size_t)FFT_STOCK_SMEM) {
        const dim3 grid2((unsigned)((nlines + Ls - 1) / Ls));
        const int nt = std::max(32, std::min(1024, Ls * a.M / 4));
        if (a.pow2)
            fft_lines_stockham_kernel<true, COLS><<<grid2, nt, sm2, st>>>(
                X, a.n, a.M, a.log2M, Ls, elem_stride, line_stride, nlines, a.tw, a.chirp, B,
                inverse ? 1 : 0, mask, mscale);
        else
            fft_lines_stockham_kernel<false, COLS><<<grid2, nt, sm2, st>>>(
                X, a.n, a.M, a.log2M, Ls, elem_stride, line_stride, nlines, a.tw, a.chirp, B,
                inverse ? 1 : 0, mask, mscale);
        return cudaGetLastError();
    }
    if (a.pow2)
        fft_lines_kernel<true, COLS><<<grid, FFT_THREADS, sm, st>>>(
            X, a.n, a.M, a.log2M, L, elem_stride, line_stride, nlines, a.tw, a.chirp, B,
            inverse ? 1 : 0, mask, mscale);
    else
        fft_lines_kernel<false, COLS><<<grid, FFT_THREADS, sm, st>>>(
            X, a.n, a.M, a.log2M, L, elem_stride, line_stride, nlines, a.tw, a.chirp, B,
            inverse ? 1 : 0, mask, mscale);
    return cudaGetLastError();
}

cudaError_t fft2d(const FftPlan& p, float2* X, bool inverse, cudaStream_t st, const uint8_t* mask,
                  float mscale) {
    if (!p.rows || !p.cols) return cudaErrorInvalidValue;
    // a line of length 1 is its own transform; the mask goes with the last
    // pass (the columns, or the rows of a one-row image)
    cudaError_t e = cudaSuccess;
    const bool cols = p.H > 1;
    if (p.W > 1)
        e = lines<false>(*p.rows, X, 1, p.W, p.H, inverse, st, cols ? nullptr : mask, mscale);
    if (e == cudaSuccess && cols) e = lines<true>(*p.cols, X, p.W, 1, p.W, inverse, st, mask, mscale);
    if (e == cudaSuccess && mask && p.H == 1 && p.W == 1)   // no pass ran: a 1 x 1 image
        e = cudaErrorInvalidValue;
    return e;
}

}  // namespace cm
