// Image-domain steps: lambda (Sec. "Parameter settings"), the closed-form
// image estimation for a periodic blur (Eq. 6, diagonal in the Fourier
// domain, cuFFT transforms + own pointwise kernels), and the initialisation
// of inverse problems, x0 = (A^T A + c L)^-1 A^T y with c = 0.2 sigma^2 / lambda
// and L the periodic 5-point negative Laplacian (FFT for a blur, conjugate
// gradients for a pixelwise A).
#include "epll_internal.cuh"

#include <cooperative_groups.h>

namespace epll {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs

// ---------------------------------------------------------------- compensated FP32 sums
// Sums of many FP32 terms are carried as unevaluated pairs (s, c) of floats:
// every addition is an exact TwoSum (Knuth) whose rounding error goes into c,
// and a product's rounding error is recovered exactly with one FMA, as in the
// Dot2 algorithm of Ogita, Rump & Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 2005).  The result is about as accurate as if the sum
// had been formed in twice the working precision.  Intrinsics keep the
// compiler from contracting or reordering these operations.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void csum_add(float &s, float &c, float v)
{
    float t, e;
    two_sum(s, v, t, e);
    s = t;
    c = __fadd_rn(c, e);
}
// s += u * v with the product's rounding error kept
__device__ __forceinline__ void csum_fma(float &s, float &c, float u, float v)
{
    const float p = __fmul_rn(u, v);
    const float pe = __fmaf_rn(u, v, -p);
    csum_add(s, c, p);
    c = __fadd_rn(c, pe);
}
__device__ __forceinline__ void csum_merge(float &s, float &c, float s2, float c2)
{
    float t, e;
    two_sum(s, s2, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, e));
}
// (s, c) / d for a float d > 0: quotient with one correction step
__device__ __forceinline__ void csum_div(float s, float c, float d, float &q, float &ql)
{
    q = __fdiv_rn(s, d);
    const float rem = __fadd_rn(__fmaf_rn(-q, d, s), c);
    ql = __fdiv_rn(rem, d);
}

// Block-wide sum of (s, c) pairs and maximum m, in a fixed order; the result
// is valid in thread 0.
template <int NT>
__device__ void block_csum_max(float &s, float &c, float &m)
{
    __shared__ float ws_[NT / 32][3];
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, s, o), c2 = __shfl_down_sync(0xffffffffu, c, o);
        const float m2 = __shfl_down_sync(0xffffffffu, m, o);
        csum_merge(s, c, s2, c2);
        m = fmaxf(m, m2);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { ws_[wid][0] = s; ws_[wid][1] = c; ws_[wid][2] = m; }
    __syncthreads();
    if (wid == 0) {
        s = lane < NT / 32 ? ws_[lane][0] : 0.0f;
        c = lane < NT / 32 ? ws_[lane][1] : 0.0f;
        m = lane < NT / 32 ? ws_[lane][2] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s, o), c2 = __shfl_down_sync(0xffffffffu, c, o);
            const float m2 = __shfl_down_sync(0xffffffffu, m, o);
            csum_merge(s, c, s2, c2);
            m = fmaxf(m, m2);
        }
    }
}

// ---------------------------------------------------------------- lambda
// Partials of (sum of squared operator eigenvalues squared, max squared
// eigenvalue): mode 1 over the gains a (A = diag(a)); mode 2 over the half
// spectrum of the blur (weights 2 for the columns that stand for two
// frequencies of the full spectrum); mode 3 over the low-resolution
// frequencies of a blur followed by decimation by d, whose eigenvalues are
// the per-block values e (full complex spectrum Hh).  Partial b:
// part[3b..3b+2] = (s, c, max).
__global__ void __launch_bounds__(RED_THREADS)
k_lambda_part(int mode, const float *__restrict__ a, const cufftComplex *__restrict__ Hh, int H,
              int W, int d, float *__restrict__ part)
{
    float s = 0.0f, c = 0.0f, m = 0.0f;
    const int Wc = W / 2 + 1;
    const int h = H / d, w = W / d;
    const int total = mode == 1 ? H * W : mode == 2 ? H * Wc : h * w;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
        float e2, wgt = 1.0f;
        if (mode == 1) {
            const float v = a[p];
            e2 = __fmul_rn(v, v);
        } else if (mode == 3) {
            // the one non-zero eigenvalue of the block of A^T A at this
            // low-resolution frequency: d^-2 sum over its aliases of |H|^2
            const int u0 = p / w, v0 = p % w;
            float es = 0.0f, ec = 0.0f;
            for (int ia = 0; ia < d; ++ia)
                for (int ib = 0; ib < d; ++ib) {
                    const cufftComplex z = Hh[(size_t)(u0 + ia * h) * W + (v0 + ib * w)];
                    csum_fma(es, ec, z.x, z.x);
                    csum_fma(es, ec, z.y, z.y);
                }
            e2 = __fadd_rn(es, ec) / (float)(d * d);
        } else {
            const int col = p % Wc;
            const float re = Hh[p].x, im = Hh[p].y;
            e2 = __fmaf_rn(re, re, __fmul_rn(im, im));
            if (col != 0 && !(W % 2 == 0 && col == W / 2)) wgt = 2.0f;
        }
        // e2^2 with its rounding error, times the (exact) weight
        const float p4 = __fmul_rn(e2, e2), p4e = __fmaf_rn(e2, e2, -p4);
        csum_add(s, c, wgt * p4);
        c = __fadd_rn(c, wgt * p4e);
        m = fmaxf(m, e2);
    }
    block_csum_max<RED_THREADS>(s, c, m);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = s;
        part[3 * blockIdx.x + 1] = c;
        part[3 * blockIdx.x + 2] = m;
    }
}

// lambda = min{ N^-1 sum / max , 250 sigma_255^2 }; mode 0 = denoising (value 1).
// Writes lamf[0..1] = lambda as an unevaluated float pair and d_lambda[0] =
// their sum, the input of the (FP64) per-beta tables.
__global__ void __launch_bounds__(RED_THREADS)
k_lambda_final(int mode, const float *__restrict__ part, int nparts, float N, float cap_hi,
               float cap_lo, float *__restrict__ lamf, double *__restrict__ d_lambda)
{
    float s = 0.0f, c = 0.0f, m = 0.0f;
    if (mode != 0)
        for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
            csum_merge(s, c, part[3 * b], part[3 * b + 1]);
            m = fmaxf(m, part[3 * b + 2]);
        }
    block_csum_max<RED_THREADS>(s, c, m);
    if (threadIdx.x == 0) {
        float v = 1.0f, vl = 0.0f;
        if (mode != 0) {
            float q, ql;
            csum_div(s, c, N, q, ql);
            two_sum(q, ql, q, ql);
            csum_div(q, ql, m, v, vl);
            two_sum(v, vl, v, vl);
        }
        if (v > cap_hi || (v == cap_hi && vl > cap_lo)) { v = cap_hi; vl = cap_lo; }
        lamf[0] = v;
        lamf[1] = vl;
        d_lambda[0] = (double)v + (double)vl;
    }
}

static void split_float(double v, float *hi, float *lo)
{
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
}

epll_status launch_lambda(epll_gmm *g, int kind, const float *a, int H, int W, double sigma,
                          cudaStream_t st, int d)
{
    Workspace &ws = g->ws;
    const double s255 = 255.0 * sigma;
    float cap_hi, cap_lo;
    split_float(250.0 * s255 * s255, &cap_hi, &cap_lo);
    float *part = ws.red;
    if (kind == EPLL_DENOISE) {
        k_lambda_final<<<1, RED_THREADS, 0, st>>>(0, part, 0, (float)H * (float)W, cap_hi, cap_lo, ws.lamf,
                                                 ws.scal);
        EPLL_LAUNCHED(g);
        return EPLL_OK;
    }
    const int mode = kind == EPLL_PIXELWISE ? 1 : kind == EPLL_CONV_PERIODIC ? 2 : 3;
    k_lambda_part<<<RED_BLOCKS, RED_THREADS, 0, st>>>(mode, a, ws.Hh, H, W, d, part);
    EPLL_LAUNCHED(g);
    k_lambda_final<<<1, RED_THREADS, 0, st>>>(mode, part, RED_BLOCKS, (float)((double)H * W), cap_hi, cap_lo,
                                             ws.lamf, ws.scal);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

// ---------------------------------------------------------------- FFT path
__global__ void k_wrap_kernel(const float *__restrict__ kern, int kh, int kw, int H, int W,
                              float *__restrict__ out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kh * kw) return;
    const int u = q / kw, v = q % kw;
    const int i = ((u - kh / 2) % H + H) % H, j = ((v - kw / 2) % W + W) % W;
    atomicAdd(&out[(size_t)i * W + j], kern[q]);
}

// x0 = conj(H) Y / (|H|^2 + c Lhat), c = 0.2 sigma^2 / lambda; 1/N of the inverse folded in.
__global__ void k_fft_init(const cufftComplex *__restrict__ Hh, const cufftComplex *__restrict__ Yh,
                           int H, int W, float c_num, const float *__restrict__ lamf,
                           cufftComplex *__restrict__ X)
{
    const int Wc = W / 2 + 1;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * Wc) return;
    const int u = p / Wc, v = p % Wc;
    const float c = c_num / lamf[0];
    const float Lh = 4.0f - 2.0f * cospif(2.0f * (float)u / (float)H) - 2.0f * cospif(2.0f * (float)v / (float)W);
    const cufftComplex h = Hh[p], y = Yh[p];
    const float h2 = h.x * h.x + h.y * h.y;
    const float inv = 1.0f / ((h2 + c * Lh) * (float)H * (float)W);
    X[p] = make_float2((h.x * y.x + h.y * y.y) * inv, (h.x * y.y - h.y * y.x) * inv);
}

// X = (conj(H) Y + bs X) / (|H|^2 + bs), bs = lambda * mult
__global__ void k_fft_update(const cufftComplex *__restrict__ Hh, const cufftComplex *__restrict__ Yh,
                             int H, int W, const float *__restrict__ lamf, float bmult,
                             cufftComplex *__restrict__ X)
{
    const int Wc = W / 2 + 1;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * Wc) return;
    const float bs = lamf[0] * bmult;
    const cufftComplex h = Hh[p], y = Yh[p], x = X[p];
    const float h2 = h.x * h.x + h.y * h.y;
    const float inv = 1.0f / ((h2 + bs) * (float)H * (float)W);
    X[p] = make_float2((h.x * y.x + h.y * y.y + bs * x.x) * inv, (h.x * y.y - h.y * y.x + bs * x.y) * inv);
}

#define EPLL_FFT(call)                                                               \
    do {                                                                             \
        cufftResult r_ = (call);                                                     \
        if (r_ != CUFFT_SUCCESS) {                                                   \
            set_error(std::string(#call) + " failed with cufftResult " + std::to_string((int)r_)); \
            return EPLL_ECUDA;                                                       \
        }                                                                            \
    } while (0)

epll_status fft_prepare(epll_gmm *g, const float *kernel, int kh, int kw, const float *y,
                        int H, int W, cudaStream_t st, bool kernel_dev)
{
    Workspace &ws = g->ws;
    int slot = -1;
    for (int i = 0; i < ws.nplans; ++i)
        if (ws.plan_h[i] == H && ws.plan_w[i] == W) slot = i;
    if (slot < 0) {
        if (ws.nplans == Workspace::FFT_CACHE) {  // drop the oldest size
            cufftDestroy(ws.plan_fw[0]);
            cufftDestroy(ws.plan_bw[0]);
            for (int i = 1; i < ws.nplans; ++i) {
                ws.plan_h[i - 1] = ws.plan_h[i];
                ws.plan_w[i - 1] = ws.plan_w[i];
                ws.plan_fw[i - 1] = ws.plan_fw[i];
                ws.plan_bw[i - 1] = ws.plan_bw[i];
            }
            --ws.nplans;
        }
        cufftHandle fw = 0, bw = 0;
        EPLL_FFT(cufftPlan2d(&fw, H, W, CUFFT_R2C));
        cufftResult r = cufftPlan2d(&bw, H, W, CUFFT_C2R);
        if (r != CUFFT_SUCCESS) {
            cufftDestroy(fw);
            set_error("cufftPlan2d (C2R) failed with cufftResult " + std::to_string((int)r));
            return EPLL_ECUDA;
        }
        slot = ws.nplans++;
        ws.plan_h[slot] = H;
        ws.plan_w[slot] = W;
        ws.plan_fw[slot] = fw;
        ws.plan_bw[slot] = bw;
    }
    ws.plan_r2c = ws.plan_fw[slot];
    ws.plan_c2r = ws.plan_bw[slot];
    EPLL_FFT(cufftSetStream(ws.plan_r2c, st));
    EPLL_FFT(cufftSetStream(ws.plan_c2r, st));
    const size_t N = (size_t)H * W;
    const float *dk = kernel;
    if (!kernel_dev) {
        // stage the small kernel through the CG buffer (kh*kw <= N floats)
        EPLL_CU(cudaMemcpyAsync(ws.cg, kernel, sizeof(float) * (size_t)kh * kw, cudaMemcpyHostToDevice, st));
        dk = ws.cg;
    }
    EPLL_CU(cudaMemsetAsync(ws.kern, 0, sizeof(float) * N, st));
    k_wrap_kernel<<<(kh * kw + 255) / 256, 256, 0, st>>>(dk, kh, kw, H, W, ws.kern);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecR2C(ws.plan_r2c, ws.kern, ws.Hh));
    EPLL_FFT(cufftExecR2C(ws.plan_r2c, const_cast<float *>(y), ws.Yh));
    return EPLL_OK;
}

epll_status fft_init(epll_gmm *g, int H, int W, double sigma, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int M = H * (W / 2 + 1);
    k_fft_init<<<(M + 255) / 256, 256, 0, st>>>(ws.Hh, ws.Yh, H, W, (float)(0.2 * sigma * sigma), ws.lamf, ws.Xh);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecC2R(ws.plan_c2r, ws.Xh, ws.xhat));
    return EPLL_OK;
}

epll_status fft_update(epll_gmm *g, int H, int W, double bmult, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int M = H * (W / 2 + 1);
    EPLL_FFT(cufftExecR2C(ws.plan_r2c, ws.xtil, ws.Xh));
    k_fft_update<<<(M + 255) / 256, 256, 0, st>>>(ws.Hh, ws.Yh, H, W, ws.lamf, (float)bmult, ws.Xh);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecC2R(ws.plan_c2r, ws.Xh, ws.xhat));
    return EPLL_OK;
}

// ---------------------------------------------------------------- weighted update (`valid` boundary)
// With the `valid` boundary the patch overlap of Eq. 6 varies over the image,
// so the periodic-blur update (H^T H + bs diag(w)) x = H^T y + bs w xtil is
// not diagonal in any Fourier basis: it is solved by conjugate gradients from
// x = xtil (residual H^T (y - H xtil)), H^T H applied through the R2C / C2R
// transforms of the FFT path, dot products as compensated FP32 block partials
// reduced by one block in a fixed order.  Scalars sc: rr, alpha, beta, done.
__global__ void k_cgw_r0(const cufftComplex *__restrict__ Hh, const cufftComplex *__restrict__ Yh, int M,
                         float invN, cufftComplex *__restrict__ X)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const cufftComplex h = Hh[p], x = X[p], y = Yh[p];
    const float er = y.x - (h.x * x.x - h.y * x.y), ei = y.y - (h.x * x.y + h.y * x.x);
    X[p] = make_float2((h.x * er + h.y * ei) * invN, (h.x * ei - h.y * er) * invN);  // conj(H) e / N
}

__global__ void k_cgw_h2(const cufftComplex *__restrict__ Hh, int M, float invN, cufftComplex *__restrict__ X)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const cufftComplex h = Hh[p], x = X[p];
    const float g = (h.x * h.x + h.y * h.y) * invN;
    X[p] = make_float2(x.x * g, x.y * g);
}

// q += bs w d; partial d^T q
__global__ void __launch_bounds__(RED_THREADS)
k_cgw_q(float *__restrict__ q, const float *__restrict__ d, const float *__restrict__ w,
        const float *__restrict__ lamf, float bmult, int N, float *__restrict__ part)
{
    const float bs = lamf[0] * bmult;
    float s = 0.0f, c = 0.0f, m = 0.0f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const float dv = d[p];
        const float qv = fmaf(bs * w[p], dv, q[p]);
        q[p] = qv;
        csum_fma(s, c, dv, qv);
    }
    block_csum_max<RED_THREADS>(s, c, m);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s;
        part[2 * blockIdx.x + 1] = c;
    }
}

// partial r^T r, or (x, r updated first unless done) after x += alpha d, r -= alpha q
__global__ void __launch_bounds__(RED_THREADS)
k_cgw_xr(float *__restrict__ x, float *__restrict__ r, const float *__restrict__ d, const float *__restrict__ q,
         const float *__restrict__ sc, int N, int update, float *__restrict__ part)
{
    const bool go = update && sc[3] == 0.0f;
    const float alpha = sc[1];
    float s = 0.0f, c = 0.0f, m = 0.0f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        float rv = r[p];
        if (go) {
            x[p] = fmaf(alpha, d[p], x[p]);
            rv = fmaf(-alpha, q[p], rv);
            r[p] = rv;
        }
        csum_fma(s, c, rv, rv);
    }
    block_csum_max<RED_THREADS>(s, c, m);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s;
        part[2 * blockIdx.x + 1] = c;
    }
}

// which 0: rr = sum (done if not positive); 1: dq = sum, alpha = rr / dq
// (done if dq is not positive); 2: beta = sum / rr, rr = sum (done if not positive)
__global__ void __launch_bounds__(RED_THREADS)
k_cgw_scalar(int which, const float *__restrict__ part, int nparts, float *__restrict__ sc)
{
    float s = 0.0f, c = 0.0f, m = 0.0f;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) csum_merge(s, c, part[2 * b], part[2 * b + 1]);
    block_csum_max<RED_THREADS>(s, c, m);
    if (threadIdx.x) return;
    const float v = __fadd_rn(s, c);
    if (which == 0) {
        sc[0] = v;
        sc[3] = v > 0.0f ? 0.0f : 1.0f;
    } else if (sc[3] == 0.0f) {
        if (which == 1) {
            if (!(v > 0.0f)) sc[3] = 1.0f;
            else sc[1] = sc[0] / v;
        } else {
            sc[2] = v / sc[0];
            sc[0] = v;
            if (!(v > 0.0f)) sc[3] = 1.0f;
        }
    }
}

__global__ void k_cgw_d(float *__restrict__ d, const float *__restrict__ r, const float *__restrict__ sc, int N)
{
    if (sc[3] != 0.0f) return;
    const float beta = sc[2];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) d[p] = fmaf(beta, d[p], r[p]);
}

epll_status cgw_update(epll_gmm *g, int H, int W, double bmult, int iters, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const size_t cap = ws.capN;
    const int N = H * W, M = H * (W / 2 + 1);
    const float invN = 1.0f / ((float)H * (float)W);
    float *r = ws.cg, *dd = ws.cg + cap, *q = ws.cg + 2 * cap;
    float *part = ws.red, *sc = ws.lamf + 4;
    EPLL_CU(cudaMemcpyAsync(ws.xhat, ws.xtil, sizeof(float) * (size_t)N, cudaMemcpyDeviceToDevice, st));
    EPLL_FFT(cufftExecR2C(ws.plan_r2c, ws.xtil, ws.Xh));
    k_cgw_r0<<<(M + 255) / 256, 256, 0, st>>>(ws.Hh, ws.Yh, M, invN, ws.Xh);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecC2R(ws.plan_c2r, ws.Xh, r));
    k_cgw_xr<<<RED_BLOCKS, RED_THREADS, 0, st>>>(ws.xhat, r, dd, q, sc, N, 0, part);
    EPLL_LAUNCHED(g);
    k_cgw_scalar<<<1, RED_THREADS, 0, st>>>(0, part, RED_BLOCKS, sc);
    EPLL_LAUNCHED(g);
    EPLL_CU(cudaMemcpyAsync(dd, r, sizeof(float) * (size_t)N, cudaMemcpyDeviceToDevice, st));
    const float bm = (float)bmult;
    for (int it = 0; it < iters; ++it) {
        EPLL_FFT(cufftExecR2C(ws.plan_r2c, dd, ws.Xh));
        k_cgw_h2<<<(M + 255) / 256, 256, 0, st>>>(ws.Hh, M, invN, ws.Xh);
        EPLL_LAUNCHED(g);
        EPLL_FFT(cufftExecC2R(ws.plan_c2r, ws.Xh, q));
        k_cgw_q<<<RED_BLOCKS, RED_THREADS, 0, st>>>(q, dd, ws.wgt, ws.lamf, bm, N, part);
        EPLL_LAUNCHED(g);
        k_cgw_scalar<<<1, RED_THREADS, 0, st>>>(1, part, RED_BLOCKS, sc);
        EPLL_LAUNCHED(g);
        k_cgw_xr<<<RED_BLOCKS, RED_THREADS, 0, st>>>(ws.xhat, r, dd, q, sc, N, 1, part);
        EPLL_LAUNCHED(g);
        k_cgw_scalar<<<1, RED_THREADS, 0, st>>>(2, part, RED_BLOCKS, sc);
        EPLL_LAUNCHED(g);
        k_cgw_d<<<RED_BLOCKS, RED_THREADS, 0, st>>>(dd, r, sc, N);
        EPLL_LAUNCHED(g);
    }
    return EPLL_OK;
}

// ---------------------------------------------------------------- super-resolution
// A = S B (blur, then keep pixel (d i, d j)).  In the Fourier basis A^T A is
// block diagonal: the block at a low-resolution frequency w' couples the d^2
// high-resolution frequencies w'_k = w' + (a H/d, b W/d) that alias onto it and
// equals s g g^H with s = d^-2 and g_k = conj(B(w'_k)), while
// F(A^T y)(w'_k) = g_k Y(w'), Y the transform of the low-resolution
// observation.  Each block is solved in closed form (a rank-one update of a
// diagonal, as in Zhao et al., "Fast single image super-resolution using a
// new analytical solution for l2-l2 problems", IEEE TIP 2016):
//  - image update, (s g g^H + bs I) X = g Y + bs Xt (Woodbury):
//      X_k = Xt_k + g_k (Y - s g^H Xt) / (bs + s |g|^2);
//  - initialisation, (s g g^H + D) X = g Y with D_k = c L(w'_k) >= 0
//    (Sherman-Morrison, arranged so that no term is divided by a vanishing
//    D; D vanishes only at the zero frequency, where g_0 = 1):
//      X_k = g_k Y / (D_k + s (|g_k|^2 + sum_{j != k} |g_j|^2 D_k / D_j)),
//    X_k = 0 when some other D_j of the block is zero.
// Transforms are full complex (C2C) at both resolutions; the inverse's 1/N
// is folded into the solve.
__device__ __forceinline__ float neg_lap_symbol(int u, int v, int H, int W)
{
    return 4.0f - 2.0f * cospif(2.0f * (float)u / (float)H) - 2.0f * cospif(2.0f * (float)v / (float)W);
}

__global__ void k_real_to_complex(const float *__restrict__ x, int N, cufftComplex *__restrict__ out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) out[p] = make_float2(x[p], 0.0f);
}

__global__ void k_real_part(const cufftComplex *__restrict__ X, int N, float *__restrict__ out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) out[p] = X[p].x;
}

// mode 0: initialisation (c = c_num / lambda); mode 1: image update (bs = lambda * bmult, X holds Xt)
__global__ void k_sr_solve(int mode, const cufftComplex *__restrict__ Hh, const cufftComplex *__restrict__ Yl,
                           cufftComplex *__restrict__ X, int H, int W, int d, float c_num,
                           const float *__restrict__ lamf, float bmult)
{
    const int h = H / d, w = W / d;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= h * w) return;
    const int u0 = q / w, v0 = q % w;
    const float s = 1.0f / (float)(d * d);
    const float invN = 1.0f / ((float)H * (float)W);
    const cufftComplex Y = Yl[q];
    const int nk = d * d;
    auto at = [&](int k) { return (size_t)(u0 + (k / d) * h) * W + (v0 + (k % d) * w); };
    if (mode == 0) {
        const float c = c_num / lamf[0];
        for (int k = 0; k < nk; ++k) {
            const size_t pk = at(k);
            const cufftComplex hk = Hh[pk];
            const float Dk = c * neg_lap_symbol(u0 + (k / d) * h, v0 + (k % d) * w, H, W);
            float den = hk.x * hk.x + hk.y * hk.y;
            bool zero = false;
            for (int j = 0; j < nk; ++j) {
                if (j == k) continue;
                const float Dj = c * neg_lap_symbol(u0 + (j / d) * h, v0 + (j % d) * w, H, W);
                if (Dj == 0.0f) { zero = true; break; }
                const cufftComplex hj = Hh[at(j)];
                den = fmaf(hj.x * hj.x + hj.y * hj.y, Dk / Dj, den);
            }
            const float inv = zero ? 0.0f : invN / fmaf(s, den, Dk);
            // g_k Y with g_k = conj(H_k)
            X[pk] = make_float2((hk.x * Y.x + hk.y * Y.y) * inv, (hk.x * Y.y - hk.y * Y.x) * inv);
        }
    } else {
        const float bs = lamf[0] * bmult;
        // g^H Xt = sum_k H_k Xt_k, |g|^2
        float gr = 0.0f, gi = 0.0f, ng = 0.0f;
        for (int k = 0; k < nk; ++k) {
            const size_t pk = at(k);
            const cufftComplex hk = Hh[pk], xk = X[pk];
            gr += hk.x * xk.x - hk.y * xk.y;
            gi += hk.x * xk.y + hk.y * xk.x;
            ng += hk.x * hk.x + hk.y * hk.y;
        }
        const float inv = 1.0f / (bs + s * ng);
        const float tr = (Y.x - s * gr) * inv, ti = (Y.y - s * gi) * inv;
        for (int k = 0; k < nk; ++k) {
            const size_t pk = at(k);
            const cufftComplex hk = Hh[pk], xk = X[pk];
            // Xt_k + conj(H_k) t
            X[pk] = make_float2((xk.x + hk.x * tr + hk.y * ti) * invN, (xk.y + hk.x * ti - hk.y * tr) * invN);
        }
    }
}

epll_status sr_prepare(epll_gmm *g, const float *kernel_host, int kh, int kw, const float *ylow, int H, int W,
                       int d, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int h = H / d, w = W / d;
    if (ws.c2cH != H || ws.c2cW != W || ws.c2cd != d) {
        if (ws.plan_c2c) cufftDestroy(ws.plan_c2c);
        if (ws.plan_c2c_low) cufftDestroy(ws.plan_c2c_low);
        ws.plan_c2c = ws.plan_c2c_low = 0;
        ws.c2cH = ws.c2cW = ws.c2cd = 0;
        EPLL_FFT(cufftPlan2d(&ws.plan_c2c, H, W, CUFFT_C2C));
        EPLL_FFT(cufftPlan2d(&ws.plan_c2c_low, h, w, CUFFT_C2C));
        ws.c2cH = H;
        ws.c2cW = W;
        ws.c2cd = d;
    }
    EPLL_FFT(cufftSetStream(ws.plan_c2c, st));
    EPLL_FFT(cufftSetStream(ws.plan_c2c_low, st));
    const size_t N = (size_t)H * W;
    float *dk = ws.cg;  // scratch: kh*kw <= N floats
    EPLL_CU(cudaMemcpyAsync(dk, kernel_host, sizeof(float) * (size_t)kh * kw, cudaMemcpyHostToDevice, st));
    EPLL_CU(cudaMemsetAsync(ws.kern, 0, sizeof(float) * N, st));
    k_wrap_kernel<<<(kh * kw + 255) / 256, 256, 0, st>>>(dk, kh, kw, H, W, ws.kern);
    EPLL_LAUNCHED(g);
    k_real_to_complex<<<(int)((N + 255) / 256), 256, 0, st>>>(ws.kern, (int)N, ws.Hh);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecC2C(ws.plan_c2c, ws.Hh, ws.Hh, CUFFT_FORWARD));
    const int n = h * w;
    k_real_to_complex<<<(n + 255) / 256, 256, 0, st>>>(ylow, n, ws.Yh);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecC2C(ws.plan_c2c_low, ws.Yh, ws.Yh, CUFFT_FORWARD));
    return EPLL_OK;
}

epll_status sr_init(epll_gmm *g, int H, int W, int d, double sigma, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int n = (H / d) * (W / d), N = H * W;
    k_sr_solve<<<(n + 127) / 128, 128, 0, st>>>(0, ws.Hh, ws.Yh, ws.Xh, H, W, d, (float)(0.2 * sigma * sigma),
                                                ws.lamf, 0.0f);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecC2C(ws.plan_c2c, ws.Xh, ws.Xh, CUFFT_INVERSE));
    k_real_part<<<(N + 255) / 256, 256, 0, st>>>(ws.Xh, N, ws.xhat);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

epll_status sr_update(epll_gmm *g, int H, int W, int d, double bmult, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int n = (H / d) * (W / d), N = H * W;
    k_real_to_complex<<<(N + 255) / 256, 256, 0, st>>>(ws.xtil, N, ws.Xh);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecC2C(ws.plan_c2c, ws.Xh, ws.Xh, CUFFT_FORWARD));
    k_sr_solve<<<(n + 127) / 128, 128, 0, st>>>(1, ws.Hh, ws.Yh, ws.Xh, H, W, d, 0.0f, ws.lamf, (float)bmult);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecC2C(ws.plan_c2c, ws.Xh, ws.Xh, CUFFT_INVERSE));
    k_real_part<<<(N + 255) / 256, 256, 0, st>>>(ws.Xh, N, ws.xhat);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

// ---------------------------------------------------------------- CG path
// Conjugate gradients on (diag(a^2) + c L) x = a y from x = a y, a fixed
// number of iterations; stops early only once r^T r or d^T q is no longer
// positive.  The whole iteration runs in one launch of one thread-block
// cluster (16 CTAs where the device allows it, else 8): the CTAs split the
// pixels, and every dot product is a compensated FP32 sum (Dot2) reduced
// across the cluster through distributed shared memory, in a fixed order, so
// that every CTA obtains bit-identical step sizes.  The hardware cluster
// barrier orders the stencil's neighbour reads after their writes.  The
// search direction is recomputed on the fly (d = r + beta d_old at the pixel
// and its four neighbours) into a second buffer, so each iteration needs two
// barriers: one per dot product.
constexpr int CG_THREADS = 1024;

__device__ __forceinline__ float cg_dir(const float *__restrict__ r, const float *__restrict__ dold, float beta,
                                        bool first, size_t p)
{
    return first ? r[p] : __fmaf_rn(beta, dold[p], r[p]);
}

// Sum of the cluster's (s, c) pairs; every thread of every CTA returns the
// same float (hi + lo rounded).  `slot` alternates between calls so that a
// CTA never overwrites a partial that another CTA may still be reading.
__device__ float cluster_total(cooperative_groups::cluster_group &cl, float (*part)[2], int slot, float s,
                               float c)
{
    __shared__ float wsum[CG_THREADS / 32][2];
    __shared__ float total;
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, s, o), c2 = __shfl_down_sync(0xffffffffu, c, o);
        csum_merge(s, c, s2, c2);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { wsum[wid][0] = s; wsum[wid][1] = c; }
    __syncthreads();
    if (wid == 0) {
        s = wsum[lane][0];
        c = wsum[lane][1];
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s, o), c2 = __shfl_down_sync(0xffffffffu, c, o);
            csum_merge(s, c, s2, c2);
        }
        if (lane == 0) { part[slot][0] = s; part[slot][1] = c; }
    }
    cl.sync();
    if (wid == 0) {
        const int nb = (int)cl.num_blocks();
        s = 0.0f;
        c = 0.0f;
        if (lane < nb) {
            const float *rp = cl.map_shared_rank(&part[slot][0], lane);
            s = rp[0];
            c = rp[1];
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s, o), c2 = __shfl_down_sync(0xffffffffu, c, o);
            csum_merge(s, c, s2, c2);
        }
        if (lane == 0) total = __fadd_rn(s, c);
    }
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(CG_THREADS, 1)
k_cg_cluster(const float *__restrict__ a, const float *__restrict__ y, int H, int W, float c_num,
             const float *__restrict__ lamf, int iters, float *__restrict__ x, float *__restrict__ r,
             float *__restrict__ d0, float *__restrict__ d1, float *__restrict__ q)
{
    namespace cgx = cooperative_groups;
    cgx::cluster_group cl = cgx::this_cluster();
    __shared__ float part[2][2];
    const int rank = (int)cl.block_rank(), nb = (int)cl.num_blocks();
    const size_t N = (size_t)H * W;
    const size_t chunk = (N + nb - 1) / nb;
    const size_t p0 = (size_t)rank * chunk, p1 = p0 + chunk < N ? p0 + chunk : N;
    const float c = c_num / lamf[0];
    const float c4 = 4.0f * c;
    for (size_t p = p0 + threadIdx.x; p < p1; p += CG_THREADS) x[p] = a[p] * y[p];
    cl.sync();
    // r = a y - (diag(a^2) + c L) x, rr = r^T r
    float s = 0.0f, e = 0.0f;
    for (size_t p = p0 + threadIdx.x; p < p1; p += CG_THREADS) {
        const int i = (int)(p / W), j = (int)(p % W);
        const size_t pn = (size_t)(i ? i - 1 : H - 1) * W + j, ps = (size_t)(i + 1 < H ? i + 1 : 0) * W + j;
        const size_t pw = (size_t)i * W + (j ? j - 1 : W - 1), pe = (size_t)i * W + (j + 1 < W ? j + 1 : 0);
        const float ap = a[p], xv = x[p];
        const float lap = c4 * xv - c * (x[pn] + x[ps] + x[pw] + x[pe]);
        const float rv = ap * y[p] - (ap * ap * xv + lap);
        r[p] = rv;
        csum_fma(s, e, rv, rv);
    }
    float rr = cluster_total(cl, part, 1, s, e);
    float beta = 0.0f;
    float *dold = d1, *dnew = d0;
    for (int it = 0; it < iters && rr > 0.0f; ++it) {
        const bool first = it == 0;
        // d = r + beta d_old (first: d = r), q = A d, dq = d^T q
        s = 0.0f;
        e = 0.0f;
        for (size_t p = p0 + threadIdx.x; p < p1; p += CG_THREADS) {
            const int i = (int)(p / W), j = (int)(p % W);
            const size_t pn = (size_t)(i ? i - 1 : H - 1) * W + j, ps = (size_t)(i + 1 < H ? i + 1 : 0) * W + j;
            const size_t pw = (size_t)i * W + (j ? j - 1 : W - 1), pe = (size_t)i * W + (j + 1 < W ? j + 1 : 0);
            const float dv = cg_dir(r, dold, beta, first, p);
            const float nsum = cg_dir(r, dold, beta, first, pn) + cg_dir(r, dold, beta, first, ps) +
                               cg_dir(r, dold, beta, first, pw) + cg_dir(r, dold, beta, first, pe);
            const float ap = a[p];
            const float qv = ap * ap * dv + (c4 * dv - c * nsum);
            dnew[p] = dv;
            q[p] = qv;
            csum_fma(s, e, dv, qv);
        }
        const float dq = cluster_total(cl, part, 0, s, e);
        if (!(dq > 0.0f)) break;
        const float alpha = rr / dq;
        // x += alpha d, r -= alpha q, rr' = r^T r
        s = 0.0f;
        e = 0.0f;
        for (size_t p = p0 + threadIdx.x; p < p1; p += CG_THREADS) {
            const float dv = dnew[p];
            x[p] = __fmaf_rn(alpha, dv, x[p]);
            const float rv = __fmaf_rn(-alpha, q[p], r[p]);
            r[p] = rv;
            csum_fma(s, e, rv, rv);
        }
        const float rr2 = cluster_total(cl, part, 1, s, e);
        beta = rr2 / rr;
        rr = rr2;
        float *t = dold;
        dold = dnew;
        dnew = t;
    }
    cl.sync();  // no CTA leaves while another may still read its partials
}

// Cluster size of the CG kernel: 16 CTAs where one such cluster fits, else 8.
static int cg_cluster_size()
{
    static int size = 0;
    if (size) return size;
    size = 8;
    if (cudaFuncSetAttribute(k_cg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(CG_THREADS);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_cg_cluster, &cfg) == cudaSuccess && nclusters > 0)
            size = 16;
    }
    cudaGetLastError();
    return size;
}

void cg_setup() { (void)cg_cluster_size(); }

epll_status cg_init(epll_gmm *g, const float *a, const float *y, int H, int W, double sigma,
                    int iters, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const size_t cap = ws.capN;
    float *r = ws.cg, *d0 = ws.cg + cap, *d1 = ws.cg + 2 * cap, *q = ws.cg + 3 * cap;
    const int cl = cg_cluster_size();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(CG_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    EPLL_CU(cudaLaunchKernelEx(&cfg, k_cg_cluster, a, y, H, W, (float)(0.2 * sigma * sigma),
                               (const float *)ws.lamf, iters, ws.xhat, r, d0, d1, q));
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

// ---------------------------------------------------------------- pixelwise update
// x = (a y + bs xt) / (a^2 + bs), bs = lambda * mult (a == nullptr: a = 1); the
// restoration loop fuses this into the reprojection, this standalone form
// serves epll_image_update.
__global__ void k_pixel_update(const float *__restrict__ a, const float *__restrict__ y,
                               const float *__restrict__ xt, int N, const float *__restrict__ lamf, float bmult,
                               float *__restrict__ x)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const float bs = lamf[0] * bmult;
    const float ap = a ? a[p] : 1.0f;
    x[p] = (ap * y[p] + bs * xt[p]) / (ap * ap + bs);
}

epll_status launch_pixel_update(epll_gmm *g, const float *a, const float *y, const float *xt, int H, int W,
                                double bmult, float *x, cudaStream_t st)
{
    const int N = H * W;
    k_pixel_update<<<(N + 255) / 256, 256, 0, st>>>(a, y, xt, N, g->ws.lamf, (float)bmult, x);
    EPLL_LAUNCHED(g);
    return EPLL_OK;
}

}  // namespace epll
