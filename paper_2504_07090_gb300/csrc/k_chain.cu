// HMC chain on the device (App. B): momentum draws, the accept uniform and the adaptive
// step size, with every iteration captured once as a CUDA graph.
//
// Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC 2011), a counter-based generator: ten rounds of two
// 32x32 -> 64-bit products whose halves are mixed with the other counter words and the
// key, the key bumped by two Weyl constants between rounds.  Counter = (element group,
// iteration low word, iteration high word, stream), key = the 64-bit seed; stream 0 gives
// the momentum normals (Box-Muller on pairs of 24-bit uniforms), stream 1 the accept
// uniform.  The draws depend only on (seed, iteration, element), never on the launch shape.
//
// One iteration: z ~ N(0, 1) and u from the generator at the iteration number held in
// device memory; p = L z; one trajectory of n_steps with the step size held in device
// memory (run_leapfrog, which reads eps and u from the parameter slot); then the step-size
// rule of App. B on the acceptance probability a = min(1, exp(H0 - H1)):
// eps <- eps / 1.2 if a < a_min, else min(eps0, 1.2 eps); the iteration's record is
// written and the iteration number advanced.  Nothing in the graph depends on the host.
#include <cmath>
#include <vector>

#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;   // round multipliers
constexpr uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;   // key increments

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PH_W0;
            k1 += PH_W1;
        }
        const uint32_t lo0 = PH_M0 * c.x, hi0 = __umulhi(PH_M0, c.x);
        const uint32_t lo1 = PH_M1 * c.z, hi1 = __umulhi(PH_M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// 24-bit uniform in (0, 1), exact in FP32
__device__ __forceinline__ float u24(uint32_t w) { return ((float)(w >> 8) + 0.5f) * 5.9604644775390625e-8f; }

// z[4 g + j] for element group g: Box-Muller on (u0, u1) and (u2, u3)
template <typename R>
__device__ __forceinline__ void normal4(uint4 w, R out[4])
{
    const float u[4] = {u24(w.x), u24(w.y), u24(w.z), u24(w.w)};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float r = sqrtf(-2.f * logf(u[2 * k]));
        float s, c;
        sincospif(2.f * u[2 * k + 1], &s, &c);
        out[2 * k] = (R)(r * c);
        out[2 * k + 1] = (R)(r * s);
    }
}

// n normals at iteration `it` of seed (k0, k1); with cd != NULL the key comes from cd and the
// iteration from it_src[0] (device memory: the captured chain)
template <typename R>
__global__ void k_draw_normal(long long n, uint32_t k0, uint32_t k1, unsigned long long it, const ChainDev *cd,
                              const double *__restrict__ it_src, R *__restrict__ z)
{
    if (cd) {
        k0 = cd->k0;
        k1 = cd->k1;
        it = (unsigned long long)it_src[0];
    }
    const long long ng = (n + 3) / 4;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)it, (uint32_t)(it >> 32), 0u), k0, k1);
        R v[4];
        normal4<R>(w, v);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (4 * g + j < n) z[4 * g + j] = v[j];
    }
}

__device__ __forceinline__ double accept_u(uint32_t k0, uint32_t k1, unsigned long long it)
{
    const uint4 w = philox4x32_10(make_uint4(0u, (uint32_t)it, (uint32_t)(it >> 32), 1u), k0, k1);
    return ((double)w.x + 0.5) * 2.3283064365386963e-10;   // 2^-32
}

__global__ void k_draw_uniform(long long n, uint32_t k0, uint32_t k1, unsigned long long it0, double *__restrict__ u)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        u[i] = accept_u(k0, k1, it0 + (unsigned long long)i);
}

// first kernel of a call: the trace is indexed from the iteration number the state holds now
__global__ void k_chain_begin(ChainDev *__restrict__ cd, const double *__restrict__ state) { cd->it0 = state[1]; }

// parameter slot of the trajectory: eps = state[0], u drawn at iteration state[1]
__global__ void k_chain_params(const ChainDev *__restrict__ cd, const double *__restrict__ state,
                               double *__restrict__ prm)
{
    prm[0] = state[0];
    prm[1] = accept_u(cd->k0, cd->k1, (unsigned long long)state[1]);
}

// step-size rule and the iteration record {eps used, H0, H1, accepted, a}
__global__ void k_chain_adapt(const ChainDev *__restrict__ cd, double *__restrict__ state,
                              const double *__restrict__ h, const int *__restrict__ acc)
{
    const double eps = state[0], it = state[1];
    const double H0 = h[0], H1 = h[1];
    const double a = (isfinite(H0) && isfinite(H1)) ? (H1 <= H0 ? 1.0 : exp(H0 - H1)) : 0.0;
    const double next = a < cd->a_min ? eps / 1.2 : fmin(cd->eps0, 1.2 * eps);
    const long long k = (long long)(it - cd->it0);
    if (cd->trace && k >= 0 && k < cd->ntrace) {
        double *r = cd->trace + 5 * k;
        r[0] = eps;
        r[1] = H0;
        r[2] = H1;
        r[3] = (double)acc[0];
        r[4] = a;
    }
    state[0] = next;
    state[1] = it + 1.0;
}

template <typename R>
fm_status chain_ensure(Ctx &c)
{
    FM_TRY(prepare_leapfrog<R>(c));
    if (c.ch_z) return FM_OK;
    if (cudaMalloc(&c.ch_z, c.rsz * (size_t)c.n_par) != cudaSuccess ||
        cudaMalloc(&c.ch_p, c.rsz * (size_t)c.n_par) != cudaSuccess) {
        set_error("cudaMalloc chain momentum");
        return FM_ERR_ALLOC;
    }
    c.allocs.push_back(c.ch_z);
    c.allocs.push_back(c.ch_p);
    void *d = nullptr;
    if (cudaMalloc(&d, sizeof(ChainDev) + 16 * sizeof(double)) != cudaSuccess) {
        set_error("cudaMalloc chain parameters");
        return FM_ERR_ALLOC;
    }
    c.allocs.push_back(d);
    c.ch_dev = static_cast<ChainDev *>(d);
    c.ch_h = reinterpret_cast<double *>(static_cast<char *>(d) + sizeof(ChainDev));
    c.ch_acc = reinterpret_cast<int *>(c.ch_h + 4);
    return FM_OK;
}

// the kernels of one iteration, enqueued on st (captured once into the handle's graph)
template <typename R>
fm_status chain_iteration(Ctx &c, R *q, double *state, int n_steps, cudaStream_t st)
{
    k_draw_normal<R><<<cdiv((c.n_par + 3) / 4, 256), 256, 0, st>>>(c.n_par, 0u, 0u, 0ull, c.ch_dev, state + 1,
                                                                    (R *)c.ch_z);
    FM_CK_LAUNCH();
    k_chain_params<<<1, 1, 0, st>>>(c.ch_dev, state, c.lf_prm);
    FM_CK_LAUNCH();
    FM_TRY(run_precond_apply<R>(c, 0, (const R *)c.ch_z, (R *)c.ch_p, st));
    FM_TRY(run_leapfrog<R>(c, q, (R *)c.ch_p, c.lf_prm, n_steps, c.ch_h, c.ch_acc, st));
    k_chain_adapt<<<1, 1, 0, st>>>(c.ch_dev, state, c.ch_h, c.ch_acc);
    FM_CK_LAUNCH();
    return FM_OK;
}

void chain_drop_graph(Ctx &c)
{
    if (c.ch_exec) cudaGraphExecDestroy(c.ch_exec);
    if (c.ch_graph) cudaGraphDestroy(c.ch_graph);
    c.ch_exec = nullptr;
    c.ch_graph = nullptr;
}

template <typename R>
fm_status run_chain(Ctx &c, R *q, int n_iter, int n_steps, double *state, cudaStream_t st)
{
    FM_TRY(chain_ensure<R>(c));
    // the graph holds the addresses of q and the state; seed, eps0, a_min and the trace
    // pointer are read from the handle's device block, rewritten before every call
    const bool same = c.ch_exec && c.ch_q == (void *)q && c.ch_state == state && c.ch_steps == n_steps;
    FM_CK(cudaMemcpyAsync(c.ch_dev, &c.ch_host, sizeof(ChainDev), cudaMemcpyHostToDevice, st));
    k_chain_begin<<<1, 1, 0, st>>>(c.ch_dev, state);
    FM_CK_LAUNCH();
    if (!same) {
        chain_drop_graph(c);
        // one evaluation outside the capture, so that every lazily sized buffer exists
        FM_TRY(run_chi2_grad<R>(c, q, c.lf_scal + 4, c.lf_scal, (R *)c.lf_g, st));
        FM_CK(cudaStreamSynchronize(st));
        cudaStream_t cs = nullptr;
        FM_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const bool prof = c.prof_on;          // no profiling events inside the graph
        c.prof_on = false;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        fm_status s = FM_OK;
        if (e == cudaSuccess) s = chain_iteration<R>(c, q, state, n_steps, cs);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = (e == cudaSuccess) ? cudaStreamEndCapture(cs, &g) : e;
        cudaStreamDestroy(cs);
        c.prof_on = prof;
        if (s != FM_OK || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (s != FM_OK) return s;
            return cuda_fail(e2, "chain capture", __FILE__, __LINE__);
        }
        c.ch_graph = g;
        if ((e = cudaGraphInstantiate(&c.ch_exec, g, 0)) != cudaSuccess) {
            chain_drop_graph(c);
            return cuda_fail(e, "cudaGraphInstantiate (chain)", __FILE__, __LINE__);
        }
        c.ch_q = q;
        c.ch_state = state;
        c.ch_steps = n_steps;
    }
    for (int i = 0; i < n_iter; ++i) FM_CK(cudaGraphLaunch(c.ch_exec, st));
    return FM_OK;
}

fm_status bad(const char *msg)
{
    set_error("invalid argument: %s", msg);
    return FM_ERR_INVALID_ARG;
}

}  // namespace

void chain_release(Ctx &c) { chain_drop_graph(c); }

}  // namespace fm

using namespace fm;

extern "C" {

fm_status fm_draw_normal(uint64_t seed, uint64_t iteration, int64_t n, void *dev_out, int fp64, fm_stream stream)
{
    if (n < 0 || (n > 0 && !dev_out)) return bad("n >= 0 and an output are required");
    if (n == 0) return FM_OK;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const unsigned grid = cdiv((n + 3) / 4, 256) < 4096 ? cdiv((n + 3) / 4, 256) : 4096;
    if (fp64)
        k_draw_normal<double><<<grid, 256, 0, stream>>>(n, k0, k1, iteration, nullptr, nullptr, (double *)dev_out);
    else
        k_draw_normal<float><<<grid, 256, 0, stream>>>(n, k0, k1, iteration, nullptr, nullptr, (float *)dev_out);
    FM_CK_LAUNCH();
    return FM_OK;
}

fm_status fm_draw_accept_uniform(uint64_t seed, uint64_t iteration0, int64_t n, double *dev_out, fm_stream stream)
{
    if (n < 0 || (n > 0 && !dev_out)) return bad("n >= 0 and an output are required");
    if (n == 0) return FM_OK;
    const unsigned grid = cdiv(n, 256) < 4096 ? cdiv(n, 256) : 4096;
    k_draw_uniform<<<grid, 256, 0, stream>>>(n, (uint32_t)seed, (uint32_t)(seed >> 32), iteration0, dev_out);
    FM_CK_LAUNCH();
    return FM_OK;
}

fm_status fm_hmc_chain(fm_handle h, void *dev_q, int n_iter, int n_steps, double eps0, double a_min, uint64_t seed,
                       double *dev_state, double *dev_trace, fm_stream stream)
{
    if (!h) return bad("handle is NULL");
    if (!dev_q || !dev_state) return bad("dev_q and dev_state are required");
    if (n_iter < 0 || n_iter > 10000000) return bad("n_iter must be in [0, 1e7]");
    if (n_steps < 1 || n_steps > 100000) return bad("n_steps must be in [1, 100000]");
    if (!(eps0 > 0.0) || !std::isfinite(eps0)) return bad("eps0 must be > 0");
    if (!(a_min >= 0.0 && a_min <= 1.0)) return bad("a_min must be in [0, 1]");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    if (!c.have_data) { set_error("fm_set_data has not been called"); return FM_ERR_STATE; }
    if (!c.pc_chol) { set_error("fm_build_precond has not been called"); return FM_ERR_STATE; }
    c.ch_host.eps0 = eps0;
    c.ch_host.a_min = a_min;
    c.ch_host.k0 = (uint32_t)seed;
    c.ch_host.k1 = (uint32_t)(seed >> 32);
    c.ch_host.it0 = 0.0;                  // set on the device from dev_state[1]
    c.ch_host.trace = dev_trace;
    c.ch_host.ntrace = dev_trace ? n_iter : 0;
    if (c.prec == FM_PREC_FP64_SIMT) return run_chain<double>(c, (double *)dev_q, n_iter, n_steps, dev_state, stream);
    return run_chain<float>(c, (float *)dev_q, n_iter, n_steps, dev_state, stream);
}

fm_status fm_chain_kernels(fm_handle h, int64_t *out)
{
    if (!h || !out) return bad("handle and out are required");
    Ctx &c = *reinterpret_cast<Ctx *>(h);
    *out = 0;
    if (!c.ch_graph) return FM_OK;
    size_t n = 0;
    FM_CK(cudaGraphGetNodes(c.ch_graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    FM_CK(cudaGraphGetNodes(c.ch_graph, nodes.data(), &n));
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType t;
        FM_CK(cudaGraphNodeGetType(node, &t));
        if (t == cudaGraphNodeTypeKernel) ++*out;
    }
    return FM_OK;
}

}  // extern "C"
