// Patch sampling that allocates no device memory.
//
// Some callers cannot allocate device memory while they run this library:
// code that executes between a pool allocator's fixed reservations, inside
// a real-time loop where cudaMalloc's implicit synchronisation would stall
// other streams, or on a context whose memory was handed out entirely up
// front.  epll_sample, the test entry point for the patch samplers, allocates
// its radix-select scratch with cudaMalloc on every call; this variant keeps
// that scratch in a file-scope device array instead, so the caller provides
// only the output buffer.
#include "epll_internal.cuh"

#include <string>

namespace epll {

// Largest image served: 2^20 pixels (for example 1024 x 1024).
constexpr int NOALLOC_MAX_PIXELS = 1 << 20;
// Sampler scratch of that size (the layout of the allocating entry point),
// followed by the per-anchor multiplicity array.
constexpr size_t NOALLOC_SAMPLER_WORDS = sampler_words((size_t)NOALLOC_MAX_PIXELS);
constexpr size_t NOALLOC_WORDS = NOALLOC_SAMPLER_WORDS + (size_t)NOALLOC_MAX_PIXELS;

// About 4.2 MB on every device that loads the library, held until exit.
static __device__ __align__(256) unsigned g_noalloc_scratch[NOALLOC_WORDS];

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// on every call with the device current (a lookup allocates nothing; the
// first one on a device loads the library's device code there if that has
// not happened yet).
static epll_status noalloc_scratch(unsigned **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return EPLL_ECUDA;
    }
    *out = static_cast<unsigned *>(p);
    return EPLL_OK;
}

__global__ void k_noalloc_iota(int *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = i;
}

}  // namespace epll

using namespace epll;

extern "C" epll_status epll_sample_noalloc(int H, int W, const epll_options *opt, int t, int *anchors,
                                           int *n_out, void *stream)
{
    if (!anchors || !n_out) {
        set_error("epll_sample_noalloc: null output pointer");
        return EPLL_EINVAL;
    }
    epll_options o;
    if (opt) o = *opt; else epll_options_default(&o);
    epll_status s;
    if ((s = check_image(H, W))) return s;
    if ((long long)H * W > NOALLOC_MAX_PIXELS) {
        set_error("epll_sample_noalloc: image has more than 2^20 pixels, the size its static scratch serves");
        return EPLL_EINVAL;
    }
    if ((s = check_options(o, H, W))) return s;
    unsigned *scratch = nullptr;
    s = noalloc_scratch(&scratch);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)H * W;
    unsigned *mult = scratch + NOALLOC_SAMPLER_WORDS;
    epll_gmm tmp;  // carries only the launch counter; nothing is allocated
    int n = 0;
    s = launch_sample(&tmp, H, W, o, t, 1, &n, anchors, mult, scratch, sampler_stride(N), st);
    if (s) return s;
    if (o.subset == EPLL_SUBSET_ALL) {
        k_noalloc_iota<<<(n + 255) / 256, 256, 0, st>>>(anchors, n);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
            return EPLL_ECUDA;
        }
    }
    *n_out = n;
    return EPLL_OK;
}
