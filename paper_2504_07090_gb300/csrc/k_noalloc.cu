// fm_sky_pixels_noalloc: the separable mode -> pixel transform without any device
// allocation, for callers that cannot call cudaMalloc at call time -- code that runs
// under an allocator it does not own (a host framework that hands out only the tensors
// it manages), or inside a region where a new allocation would break a capture or a
// memory budget.  The caller passes every input and output; the one intermediate
// (Phi * a, n_freq x n_ra x n_mode_dec floats) lives in a file-scope device array that
// every GPU loading this library holds until the process exits.
#include <mutex>

#include "fm_internal.cuh"

#define FM_NOALLOC_MAX_SCRATCH (1 << 21)   // floats (8 MiB)

static __device__ __align__(256) float g_noalloc_scratch[FM_NOALLOC_MAX_SCRATCH];

namespace fm {
namespace {

// C[b][i][j] = sum_k A[b][i][k] B[b][k][j] with general strides, 32x32 tiles
__global__ void __launch_bounds__(256) k_noalloc_gemm(int M, int N, int K, long long sAb, long long sAi, long long sAk,
                                                      long long sBb, long long sBk, long long sBj, long long sCb,
                                                      long long sCi, long long sCj, const float *__restrict__ A,
                                                      const float *__restrict__ B, float *__restrict__ C)
{
    __shared__ float sa[32][33], sb[32][33];
    const int b = blockIdx.z, i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            const int r = e / 32, q = e % 32;
            sa[r][q] = (i0 + r < M && k0 + q < K) ? A[b * sAb + (i0 + r) * sAi + (k0 + q) * sAk] : 0.f;
            sb[r][q] = (k0 + r < K && j0 + q < N) ? B[b * sBb + (k0 + r) * sBk + (j0 + q) * sBj] : 0.f;
        }
        __syncthreads();
        for (int kk = 0; kk < 32; ++kk)
            for (int u = 0; u < 2; ++u)
                for (int v = 0; v < 2; ++v) acc[u][v] += sa[ty * 2 + u][kk] * sb[kk][tx * 2 + v];
        __syncthreads();
    }
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const int i = i0 + ty * 2 + u, j = j0 + tx * 2 + v;
            if (i < M && j < N) C[b * sCb + i * sCi + j * sCj] = acc[u][v];
        }
}

std::mutex g_mu;
float *g_scratch_dev[64] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device
// with that device current (the host-side symbol is only a stand-in for it).
fm_status scratch_ptr(float **out)
{
    int dev = 0;
    FM_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device index out of range"); return FM_ERR_UNSUPPORTED; }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        FM_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_dev[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_dev[dev];
    return FM_OK;
}

}  // namespace
}  // namespace fm

using namespace fm;

extern "C" fm_status fm_sky_pixels_noalloc(int n_freq, int n_ra, int n_dec, int n_mode_ra, int n_mode_dec,
                                           const float *dev_phi, const float *dev_leg, const float *dev_a,
                                           float *dev_x, fm_stream stream)
{
    if (n_freq < 1 || n_ra < 1 || n_dec < 1 || n_mode_ra < 1 || n_mode_dec < 1) {
        set_error("invalid argument: sizes must be >= 1");
        return FM_ERR_INVALID_ARG;
    }
    if (!dev_phi || !dev_leg || !dev_a || !dev_x) {
        set_error("invalid argument: NULL device pointer");
        return FM_ERR_INVALID_ARG;
    }
    const long long need = (long long)n_freq * n_ra * n_mode_dec;
    if (need > FM_NOALLOC_MAX_SCRATCH) {
        set_error("invalid argument: n_freq*n_ra*n_mode_dec = %lld exceeds the no-allocation scratch of %d floats",
                  need, FM_NOALLOC_MAX_SCRATCH);
        return FM_ERR_INVALID_ARG;
    }
    if ((long long)n_dec * n_ra > (1LL << 30) || (long long)n_mode_ra * n_mode_dec > (1LL << 30)) {
        set_error("invalid argument: grid too large");
        return FM_ERR_INVALID_ARG;
    }
    // both launches put n_freq on gridDim.z and 32-row tiles of n_ra (first) or n_dec (second)
    // on gridDim.y, each limited to 65535: checked here, before the first launch writes the
    // shared scratch
    if (n_freq > 65535 || cdiv(n_ra, 32) > 65535 || cdiv(n_dec, 32) > 65535) {
        set_error("invalid argument: n_freq = %d, n_ra = %d or n_dec = %d exceeds the launch grid limits "
                  "(n_freq <= 65535, n_ra and n_dec <= 65535 * 32)", n_freq, n_ra, n_dec);
        return FM_ERR_INVALID_ARG;
    }
    float *t1 = nullptr;
    FM_TRY(scratch_ptr(&t1));
    const long long npix = (long long)n_ra * n_dec, nk = (long long)n_mode_ra * n_mode_dec;
    // stage 1 fills every element of t1 that stage 2 reads, so nothing needs clearing
    // t1[f][r][n] = sum_m phi[r][m] a[f][m][n]
    dim3 g1(cdiv(n_mode_dec, 32), cdiv(n_ra, 32), n_freq);
    k_noalloc_gemm<<<g1, 256, 0, stream>>>(n_ra, n_mode_dec, n_mode_ra, 0, n_mode_ra, 1, nk, n_mode_dec, 1,
                                           (long long)n_ra * n_mode_dec, n_mode_dec, 1, dev_phi, dev_a, t1);
    FM_CK_LAUNCH();
    // x[f][d][r] = sum_n leg[d][n] t1[f][r][n]
    dim3 g2(cdiv(n_ra, 32), cdiv(n_dec, 32), n_freq);
    k_noalloc_gemm<<<g2, 256, 0, stream>>>(n_dec, n_ra, n_mode_dec, 0, n_mode_dec, 1, (long long)n_ra * n_mode_dec, 1,
                                           n_mode_dec, npix, n_ra, 1, dev_leg, t1, dev_x);
    FM_CK_LAUNCH();
    return FM_OK;
}
