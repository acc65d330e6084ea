// Batched trajectories over many independent problems (the batched uneven-problem workload of
// the HMC sampler, App. B applied to independent chains): one leapfrog trajectory per handle,
// all of them captured once as parallel branches of a single CUDA graph and replayed with one
// graph launch per call.  The step size and the accept uniform of every chain live in a
// device array that each call rewrites before the launch, so the graph stays valid.
//
// The chains share nothing but the GPU: each handle keeps its own workspace, so the branches
// run concurrently and a chain's arithmetic is exactly that of fm_leapfrog on its own.
#include <cmath>
#include <vector>

#include "fm_internal.cuh"

using namespace fm;

struct fm_batch_s {
    int n = 0, n_steps = 0;
    std::vector<Ctx *> ctx;
    std::vector<cudaStream_t> streams;   // one per chain, used only while capturing
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double *prm = nullptr;               // device [n][2]: eps, accept uniform
    std::vector<double> host_prm;
};

namespace {

void free_batch(fm_batch_s *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->joins)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    if (b->prm) cudaFree(b->prm);
    delete b;
}

fm_status bad(const char *msg)
{
    set_error("invalid argument: %s", msg);
    return FM_ERR_INVALID_ARG;
}

// one chi^2 + gradient evaluation per handle before the capture: every lazily sized
// buffer of the trajectory's kernels then exists, so the capture performs no allocation
fm_status warm(Ctx &c, void *q, cudaStream_t st)
{
    if (c.prec == FM_PREC_FP64_SIMT) {
        FM_TRY(prepare_leapfrog<double>(c));
        return run_chi2_grad<double>(c, (const double *)q, c.lf_scal + 4, c.lf_scal, (double *)c.lf_g, st);
    }
    FM_TRY(prepare_leapfrog<float>(c));
    return run_chi2_grad<float>(c, (const float *)q, c.lf_scal + 4, c.lf_scal, (float *)c.lf_g, st);
}

fm_status capture_chain(Ctx &c, void *q, void *p, const double *prm, int n_steps, double *h, int *acc,
                        cudaStream_t st)
{
    if (c.prec == FM_PREC_FP64_SIMT)
        return run_leapfrog<double>(c, (double *)q, (double *)p, prm, n_steps, h, acc, st);
    return run_leapfrog<float>(c, (float *)q, (float *)p, prm, n_steps, h, acc, st);
}

}  // namespace

extern "C" {

fm_status fm_create_batch(int n, const fm_config *cfgs, fm_handle *out)
{
    if (n < 1 || !cfgs || !out) return bad("fm_create_batch needs n >= 1, cfgs and out");
    for (int k = 0; k < n; ++k) out[k] = nullptr;
    for (int k = 0; k < n; ++k) {
        const fm_status s = fm_create(&cfgs[k], &out[k]);
        if (s != FM_OK) {
            for (int j = 0; j < k; ++j) {
                fm_destroy(out[j]);
                out[j] = nullptr;
            }
            return s;
        }
    }
    return FM_OK;
}

fm_status fm_batch_create(int n, const fm_handle *hs, void *const *dev_q, void *const *dev_p,
                          double *const *dev_h_out, int *const *dev_accepted_out, int n_steps, fm_batch *out)
{
    if (!out) return bad("out is NULL");
    *out = nullptr;
    if (n < 1 || !hs || !dev_q || !dev_p || !dev_h_out || !dev_accepted_out)
        return bad("fm_batch_create needs n >= 1 and the five pointer arrays");
    if (n_steps < 1 || n_steps > 100000) return bad("n_steps must be in [1, 100000]");
    for (int k = 0; k < n; ++k) {
        if (!hs[k] || !dev_q[k] || !dev_p[k] || !dev_h_out[k] || !dev_accepted_out[k])
            return bad("NULL handle or device pointer in the batch");
        for (int j = 0; j < k; ++j)
            if (hs[j] == hs[k]) return bad("a handle appears twice in the batch");
        const Ctx &c = *reinterpret_cast<const Ctx *>(hs[k]);
        if (!c.have_data) { set_error("batch chain %d: fm_set_data has not been called", k); return FM_ERR_STATE; }
        if (!c.pc_chol) { set_error("batch chain %d: fm_build_precond has not been called", k); return FM_ERR_STATE; }
    }
    fm_batch_s *b = new fm_batch_s;
    b->n = n;
    b->n_steps = n_steps;
    b->host_prm.assign(2 * (size_t)n, 0.0);
    auto fail = [&](fm_status s) { free_batch(b); return s; };
    auto cfail = [&](cudaError_t e, const char *what) {
        free_batch(b);
        return cuda_fail(e, what, __FILE__, __LINE__);
    };
    cudaError_t e = cudaMalloc(&b->prm, sizeof(double) * 2 * (size_t)n);
    if (e != cudaSuccess) return cfail(e, "cudaMalloc (batch parameters)");
    b->streams.assign(n, nullptr);
    b->joins.assign(n, nullptr);
    for (int k = 0; k < n; ++k) {
        if ((e = cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking)) != cudaSuccess)
            return cfail(e, "cudaStreamCreateWithFlags");
        if ((e = cudaEventCreateWithFlags(&b->joins[k], cudaEventDisableTiming)) != cudaSuccess)
            return cfail(e, "cudaEventCreateWithFlags");
        b->ctx.push_back(reinterpret_cast<Ctx *>(hs[k]));
    }
    if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess)
        return cfail(e, "cudaEventCreateWithFlags");
    for (int k = 0; k < n; ++k) {
        const fm_status s = warm(*b->ctx[k], dev_q[k], b->streams[k]);
        if (s != FM_OK) return fail(s);
    }
    for (int k = 0; k < n; ++k)
        if ((e = cudaStreamSynchronize(b->streams[k])) != cudaSuccess) return cfail(e, "cudaStreamSynchronize");

    // capture: chain k on stream k, forked from and joined back into stream 0
    cudaStream_t s0 = b->streams[0];
    if ((e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return cfail(e, "cudaStreamBeginCapture");
    fm_status st = FM_OK;
    if ((e = cudaEventRecord(b->fork, s0)) != cudaSuccess) st = cuda_fail(e, "cudaEventRecord", __FILE__, __LINE__);
    for (int k = 0; k < n && st == FM_OK; ++k) {
        cudaStream_t sk = b->streams[k];
        if (k > 0 && (e = cudaStreamWaitEvent(sk, b->fork, 0)) != cudaSuccess) {
            st = cuda_fail(e, "cudaStreamWaitEvent", __FILE__, __LINE__);
            break;
        }
        st = capture_chain(*b->ctx[k], dev_q[k], dev_p[k], b->prm + 2 * (size_t)k, n_steps, dev_h_out[k],
                           dev_accepted_out[k], sk);
        if (st != FM_OK) break;
        if (k > 0) {
            if ((e = cudaEventRecord(b->joins[k], sk)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s0, b->joins[k], 0)) != cudaSuccess)
                st = cuda_fail(e, "cudaEventRecord / cudaStreamWaitEvent", __FILE__, __LINE__);
        }
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s0, &g);
    if (st != FM_OK) {
        if (g) cudaGraphDestroy(g);
        return fail(st);
    }
    if (e != cudaSuccess) return cfail(e, "cudaStreamEndCapture");
    b->graph = g;
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) return cfail(e, "cudaGraphInstantiate");
    *out = b;
    return FM_OK;
}

fm_status fm_batch_leapfrog(fm_batch b, const double *eps, const double *u_accept, fm_stream stream)
{
    if (!b) return bad("batch is NULL");
    if (!eps || !u_accept) return bad("eps and u_accept are required");
    for (int k = 0; k < b->n; ++k) {
        if (!(eps[k] > 0.0) || !std::isfinite(eps[k])) return bad("eps must be > 0 for every chain");
        if (!(u_accept[k] >= 0.0 && u_accept[k] < 1.0)) return bad("u_accept must be in [0, 1) for every chain");
        b->host_prm[2 * (size_t)k] = eps[k];
        b->host_prm[2 * (size_t)k + 1] = u_accept[k];
    }
    // from pageable memory: the call returns once the values have been staged, so the
    // host array may change right after; the copy runs before the graph in stream order
    FM_CK(cudaMemcpyAsync(b->prm, b->host_prm.data(), sizeof(double) * 2 * (size_t)b->n, cudaMemcpyHostToDevice,
                          stream));
    FM_CK(cudaGraphLaunch(b->exec, stream));
    return FM_OK;
}

fm_status fm_batch_kernels(fm_batch b, int64_t *out)
{
    if (!b || !out) return bad("batch and out are required");
    size_t n = 0;
    FM_CK(cudaGraphGetNodes(b->graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    FM_CK(cudaGraphGetNodes(b->graph, nodes.data(), &n));
    int64_t k = 0;
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType t;
        FM_CK(cudaGraphNodeGetType(node, &t));
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    *out = k;
    return FM_OK;
}

fm_status fm_batch_destroy(fm_batch b)
{
    if (!b) return FM_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    return FM_OK;
}

}  // extern "C"
