// Image-domain steps: lambda (Sec. "Parameter settings"), the closed-form
// image estimation for a periodic blur (Eq. 6, diagonal in the Fourier
// domain, cuFFT transforms + own pointwise kernels), and the initialisation
// of inverse problems, x0 = (A^T A + c L)^-1 A^T y with c = 0.2 sigma^2 / lambda
// and L the periodic 5-point negative Laplacian (FFT for a blur, conjugate
// gradients for a pixelwise A).
#include "epll_internal.cuh"

namespace epll {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs

// ---------------------------------------------------------------- lambda
// Partials of (sum of squared operator eigenvalues squared, max squared
// eigenvalue): mode 1 over the gains a (A = diag(a)); mode 2 over the half
// spectrum of the blur (weights 2 for the columns that stand for two
// frequencies of the full spectrum).
__global__ void __launch_bounds__(RED_THREADS)
k_lambda_part(int mode, const float *__restrict__ a, const cufftComplex *__restrict__ Hh, int H,
              int W, double *__restrict__ part)
{
    __shared__ double s4[RED_THREADS], mx[RED_THREADS];
    double acc = 0.0, m = 0.0;
    const int Wc = W / 2 + 1;
    const int total = mode == 1 ? H * W : H * Wc;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
        double e2, wgt = 1.0;
        if (mode == 1) {
            double v = a[p];
            e2 = v * v;
        } else {
            const int col = p % Wc;
            const double re = Hh[p].x, im = Hh[p].y;
            e2 = re * re + im * im;
            if (col != 0 && !(W % 2 == 0 && col == W / 2)) wgt = 2.0;
        }
        acc += wgt * e2 * e2;
        m = fmax(m, e2);
    }
    s4[threadIdx.x] = acc;
    mx[threadIdx.x] = m;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            s4[threadIdx.x] += s4[threadIdx.x + s];
            mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s4[0];
        part[2 * blockIdx.x + 1] = mx[0];
    }
}

// lambda = min{ N^-1 sum / max , 250 sigma_255^2 }; mode 0 = denoising (value 1)
__global__ void __launch_bounds__(RED_THREADS)
k_lambda_final(int mode, const double *__restrict__ part, int nparts, double N, double cap,
               double *__restrict__ out)
{
    __shared__ double s4[RED_THREADS], mx[RED_THREADS];
    double acc = 0.0, m = 0.0;
    if (mode != 0)
        for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
            acc += part[2 * b];
            m = fmax(m, part[2 * b + 1]);
        }
    s4[threadIdx.x] = acc;
    mx[threadIdx.x] = m;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            s4[threadIdx.x] += s4[threadIdx.x + s];
            mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double v = mode == 0 ? 1.0 : (s4[0] / N) / mx[0];
        out[0] = v < cap ? v : cap;
    }
}

epll_status launch_lambda(epll_gmm *g, int kind, const float *a, int H, int W, double sigma,
                          cudaStream_t st)
{
    Workspace &ws = g->ws;
    const double s255 = 255.0 * sigma;
    const double cap = 250.0 * s255 * s255;
    double *part = reinterpret_cast<double *>(ws.red);
    if (kind == EPLL_DENOISE) {
        k_lambda_final<<<1, RED_THREADS, 0, st>>>(0, part, 0, (double)H * W, cap, ws.scal);
        EPLL_LAUNCHED(g);
        return EPLL_OK;
    }
    const int mode = kind == EPLL_PIXELWISE ? 1 : 2;
    k_lambda_part<<<RED_BLOCKS, RED_THREADS, 0, st>>>(mode, a, ws.Hh, H, W, part);
    EPLL_LAUNCHED(g);
    k_lambda_final<<<1, RED_THREADS, 0, st>>>(mode, part, RED_BLOCKS, (double)H * W, cap, ws.scal);
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
                           int H, int W, double sigma2, const double *__restrict__ d_lambda,
                           cufftComplex *__restrict__ X)
{
    const int Wc = W / 2 + 1;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * Wc) return;
    const int u = p / Wc, v = p % Wc;
    const float c = (float)(0.2 * sigma2 / d_lambda[0]);
    const float Lh = 4.0f - 2.0f * cospif(2.0f * (float)u / (float)H) - 2.0f * cospif(2.0f * (float)v / (float)W);
    const cufftComplex h = Hh[p], y = Yh[p];
    const float h2 = h.x * h.x + h.y * h.y;
    const float inv = 1.0f / ((h2 + c * Lh) * (float)H * (float)W);
    X[p] = make_float2((h.x * y.x + h.y * y.y) * inv, (h.x * y.y - h.y * y.x) * inv);
}

// X = (conj(H) Y + bs X) / (|H|^2 + bs), bs = lambda * mult
__global__ void k_fft_update(const cufftComplex *__restrict__ Hh, const cufftComplex *__restrict__ Yh,
                             int H, int W, const double *__restrict__ d_lambda, double bmult,
                             cufftComplex *__restrict__ X)
{
    const int Wc = W / 2 + 1;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * Wc) return;
    const float bs = (float)(d_lambda[0] * bmult);
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

epll_status fft_prepare(epll_gmm *g, const float *kernel_host, int kh, int kw, const float *y,
                        int H, int W, cudaStream_t st)
{
    Workspace &ws = g->ws;
    if (ws.planH != H || ws.planW != W) {
        if (ws.plan_r2c) cufftDestroy(ws.plan_r2c);
        if (ws.plan_c2r) cufftDestroy(ws.plan_c2r);
        ws.plan_r2c = ws.plan_c2r = 0;
        ws.planH = ws.planW = 0;
        EPLL_FFT(cufftPlan2d(&ws.plan_r2c, H, W, CUFFT_R2C));
        EPLL_FFT(cufftPlan2d(&ws.plan_c2r, H, W, CUFFT_C2R));
        ws.planH = H;
        ws.planW = W;
    }
    EPLL_FFT(cufftSetStream(ws.plan_r2c, st));
    EPLL_FFT(cufftSetStream(ws.plan_c2r, st));
    // stage the small kernel through the tail of the wrapped-kernel buffer
    const size_t N = (size_t)H * W;
    float *dk = ws.cg;  // scratch: kh*kw <= N floats
    EPLL_CU(cudaMemcpyAsync(dk, kernel_host, sizeof(float) * (size_t)kh * kw, cudaMemcpyHostToDevice, st));
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
    k_fft_init<<<(M + 255) / 256, 256, 0, st>>>(ws.Hh, ws.Yh, H, W, sigma * sigma, ws.scal, ws.Xh);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecC2R(ws.plan_c2r, ws.Xh, ws.xhat));
    return EPLL_OK;
}

epll_status fft_update(epll_gmm *g, int H, int W, double bmult, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int M = H * (W / 2 + 1);
    EPLL_FFT(cufftExecR2C(ws.plan_r2c, ws.xtil, ws.Xh));
    k_fft_update<<<(M + 255) / 256, 256, 0, st>>>(ws.Hh, ws.Yh, H, W, ws.scal, bmult, ws.Xh);
    EPLL_LAUNCHED(g);
    EPLL_FFT(cufftExecC2R(ws.plan_c2r, ws.Xh, ws.xhat));
    return EPLL_OK;
}

// ---------------------------------------------------------------- CG path
// Conjugate gradients on (diag(a^2) + c L) x = a y from x = a y, a fixed
// number of iterations; stops (device flag) once d^T q is not positive.
// Dot products: FP64 per-block partials with a fixed tree, then one block.
// scal: [0] lambda, [1] rr, [2] alpha, [3] beta, [4] done.
__device__ __forceinline__ float apply_A(const float *__restrict__ a, float c,
                                         const float *__restrict__ v, int i, int j, int H, int W)
{
    const size_t p = (size_t)i * W + j;
    const int im = i ? i - 1 : H - 1, ip = i + 1 < H ? i + 1 : 0;
    const int jm = j ? j - 1 : W - 1, jp = j + 1 < W ? j + 1 : 0;
    const float lap = 4.0f * v[p] - v[(size_t)im * W + j] - v[(size_t)ip * W + j] -
                      v[(size_t)i * W + jm] - v[(size_t)i * W + jp];
    return a[p] * a[p] * v[p] + c * lap;
}

__device__ void block_partial(double v, double *out)
{
    __shared__ double s[RED_THREADS];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(RED_THREADS)
k_cg_x0(const float *__restrict__ a, const float *__restrict__ y, int N, float *__restrict__ x)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x)
        x[p] = a[p] * y[p];
}

// r = a y - A x, d = r, partial r.r
__global__ void __launch_bounds__(RED_THREADS)
k_cg_r0(const float *__restrict__ a, const float *__restrict__ y, const float *__restrict__ x,
        int H, int W, double sigma2, const double *__restrict__ scal, float *__restrict__ r,
        float *__restrict__ d, double *__restrict__ part)
{
    const float c = (float)(0.2 * sigma2 / scal[0]);
    double acc = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < H * W; p += gridDim.x * blockDim.x) {
        const float rv = a[p] * y[p] - apply_A(a, c, x, p / W, p % W, H, W);
        r[p] = rv;
        d[p] = rv;
        acc += (double)rv * rv;
    }
    block_partial(acc, part);
}

// q = A d, partial d.q
__global__ void __launch_bounds__(RED_THREADS)
k_cg_q(const float *__restrict__ a, const float *__restrict__ d, int H, int W, double sigma2,
       const double *__restrict__ scal, float *__restrict__ q, double *__restrict__ part)
{
    const float c = (float)(0.2 * sigma2 / scal[0]);
    double acc = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < H * W; p += gridDim.x * blockDim.x) {
        const float qv = apply_A(a, c, d, p / W, p % W, H, W);
        q[p] = qv;
        acc += (double)d[p] * qv;
    }
    block_partial(acc, part);
}

// which: 0 -> rr = sum; 1 -> dq = sum, alpha = rr/dq (done if dq <= 0); 2 -> beta = sum/rr, rr = sum
__global__ void __launch_bounds__(RED_THREADS)
k_cg_scalar(int which, const double *__restrict__ part, int nparts, double *__restrict__ scal)
{
    __shared__ double s[RED_THREADS];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) acc += part[b];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x) return;
    const double v = s[0];
    if (which == 0) {
        scal[1] = v;
        scal[4] = v > 0.0 ? 0.0 : 1.0;
    } else if (which == 1) {
        if (!(v > 0.0)) scal[4] = 1.0;
        scal[2] = scal[4] != 0.0 ? 0.0 : scal[1] / v;
    } else {
        scal[3] = scal[4] != 0.0 ? 0.0 : v / scal[1];
        if (scal[4] == 0.0) scal[1] = v;
    }
}

// x += alpha d, r -= alpha q, partial r.r
__global__ void __launch_bounds__(RED_THREADS)
k_cg_xr(const float *__restrict__ d, const float *__restrict__ q, int N,
        const double *__restrict__ scal, float *__restrict__ x, float *__restrict__ r,
        double *__restrict__ part)
{
    const bool done = scal[4] != 0.0;
    const float alpha = (float)scal[2];
    double acc = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        float rv = r[p];
        if (!done) {
            x[p] = fmaf(alpha, d[p], x[p]);
            rv = fmaf(-alpha, q[p], rv);
            r[p] = rv;
        }
        acc += (double)rv * rv;
    }
    block_partial(acc, part);
}

// d = r + beta d
__global__ void __launch_bounds__(RED_THREADS)
k_cg_d(const float *__restrict__ r, int N, const double *__restrict__ scal, float *__restrict__ d)
{
    if (scal[4] != 0.0) return;
    const float b = (float)scal[3];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x)
        d[p] = fmaf(b, d[p], r[p]);
}

epll_status cg_init(epll_gmm *g, const float *a, const float *y, int H, int W, double sigma,
                    int iters, cudaStream_t st)
{
    Workspace &ws = g->ws;
    const int N = H * W;
    float *r = ws.cg, *d = ws.cg + ws.capN, *q = ws.cg + 2 * ws.capN;
    double *part = reinterpret_cast<double *>(ws.red);
    const double s2 = sigma * sigma;
    k_cg_x0<<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, y, N, ws.xhat);
    EPLL_LAUNCHED(g);
    k_cg_r0<<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, y, ws.xhat, H, W, s2, ws.scal, r, d, part);
    EPLL_LAUNCHED(g);
    k_cg_scalar<<<1, RED_THREADS, 0, st>>>(0, part, RED_BLOCKS, ws.scal);
    EPLL_LAUNCHED(g);
    for (int it = 0; it < iters; ++it) {
        k_cg_q<<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, d, H, W, s2, ws.scal, q, part);
        EPLL_LAUNCHED(g);
        k_cg_scalar<<<1, RED_THREADS, 0, st>>>(1, part, RED_BLOCKS, ws.scal);
        EPLL_LAUNCHED(g);
        k_cg_xr<<<RED_BLOCKS, RED_THREADS, 0, st>>>(d, q, N, ws.scal, ws.xhat, r, part);
        EPLL_LAUNCHED(g);
        k_cg_scalar<<<1, RED_THREADS, 0, st>>>(2, part, RED_BLOCKS, ws.scal);
        EPLL_LAUNCHED(g);
        k_cg_d<<<RED_BLOCKS, RED_THREADS, 0, st>>>(r, N, ws.scal, d);
        EPLL_LAUNCHED(g);
    }
    return EPLL_OK;
}

}  // namespace epll
