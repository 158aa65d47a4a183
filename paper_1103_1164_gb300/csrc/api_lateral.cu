// C ABI of the lateral-correction forms and of the surrogate network's trainer.
#include <math.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "dc_internal.cuh"

namespace dc {

static dc_status bad(const std::string& msg)
{
    set_error(msg);
    return DC_EINVAL;
}

static uint16_t bf16_bits(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);   // inf / nan
    u += 0x7FFFu + ((u >> 16) & 1u);                                    // round to nearest even
    return (uint16_t)(u >> 16);
}

// B fragments of mma.m16n8k16 for the three layers: for k-tile kt, n-tile nt
// and lane l, (W[k0][n], W[k0+1][n]) and (W[k0+8][n], W[k0+9][n]) as BF16 pairs
// with k0 = 16 kt + 2 (l % 4), n = 8 nt + l / 4 (zero beyond the layer's width).
void mlp_pack(const float* theta, std::vector<uint2>& frag, std::vector<float>& bias)
{
    struct Layer { int off, K, N, KT, NT; };
    const Layer L[3] = {{0, 48, 64, 3, 8}, {48 * 64 + 64, 64, 64, 4, 8}, {48 * 64 + 64 + 64 * 64 + 64, 64, 3, 4, 1}};
    frag.clear();
    for (const Layer& l : L)
        for (int kt = 0; kt < l.KT; ++kt)
            for (int nt = 0; nt < l.NT; ++nt)
                for (int lane = 0; lane < 32; ++lane) {
                    const int k0 = kt * 16 + 2 * (lane % 4), n = nt * 8 + lane / 4;
                    auto w = [&](int k) { return n < l.N ? theta[l.off + k * l.N + n] : 0.f; };
                    uint2 f;
                    f.x = (uint32_t)bf16_bits(w(k0)) | ((uint32_t)bf16_bits(w(k0 + 1)) << 16);
                    f.y = (uint32_t)bf16_bits(w(k0 + 8)) | ((uint32_t)bf16_bits(w(k0 + 9)) << 16);
                    frag.push_back(f);
                }
    bias.assign(kMlpBias, 0.f);
    const int oB1 = 48 * 64, oB2 = oB1 + 64 + 64 * 64, oB3 = oB2 + 64 + 64 * 3;
    for (int j = 0; j < 64; ++j) {
        bias[j] = theta[oB1 + j];
        bias[64 + j] = theta[oB2 + j];
    }
    for (int o = 0; o < 3; ++o) bias[128 + o] = theta[oB3 + o];
}

}  // namespace dc

using namespace dc;

struct dc_mlp {
    cudaStream_t stream = nullptr;
    float* theta = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    float* grad = nullptr;
    float* partial = nullptr;
    float* loss_part = nullptr;
    float* dX = nullptr;
    float* dT = nullptr;
    size_t cap = 0;
    int step = 0;
    int precision = DC_PRECISION_FP32;   // arithmetic of the gradient kernel
};

static const int kGradCtas = 152;

static void mlp_free(dc_mlp* m)
{
    void* b[] = {m->theta, m->m1, m->m2, m->grad, m->partial, m->loss_part, m->dX, m->dT};
    for (void* x : b)
        if (x) cudaFree(x);
    delete m;
}

extern "C" {

dc_status dc_fspb_set_surrogate(dc_plan* plan, const float* params, float rho_lo, float rho_hi)
{
    DC_NVTX("dc_fspb_set_surrogate");
    if (!plan || !params) return bad("dc_fspb_set_surrogate: NULL argument");
    if (!(rho_lo < rho_hi)) return bad("dc_fspb_set_surrogate: need rho_lo < rho_hi");
    for (int q = 0; q < kMlpParams; ++q)
        if (!isfinite(params[q])) return bad("dc_fspb_set_surrogate: non-finite parameter");
    std::vector<uint2> frag;
    std::vector<float> bias;
    mlp_pack(params, frag, bias);
    if (!plan->d_mlp_frag) DC_CUDA(dc::dev_malloc(&plan->d_mlp_frag, kMlpFragU2 * sizeof(uint2)));
    if (!plan->d_mlp_bias) DC_CUDA(dc::dev_malloc(&plan->d_mlp_bias, kMlpBias * sizeof(float)));
    DC_CUDA(cudaMemcpyAsync(plan->d_mlp_frag, frag.data(), frag.size() * sizeof(uint2), cudaMemcpyHostToDevice,
                            plan->stream));
    DC_CUDA(cudaMemcpyAsync(plan->d_mlp_bias, bias.data(), bias.size() * sizeof(float), cudaMemcpyHostToDevice,
                            plan->stream));
    plan->mlp_lo = rho_lo;
    plan->mlp_hi = rho_hi;
    plan->mlp_ready = true;
    ++plan->layout_gen;
    if (plan->lateral_mode == DC_LATERAL_MLP && plan->coeffs.density_correction) DC_CUDA(launch_lateral(plan));
    if (plan->sp_ready) plan->spmm_invalidate();
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    return DC_OK;
}

dc_status dc_fspb_set_lateral_mode(dc_plan* plan, int32_t mode)
{
    DC_NVTX("dc_fspb_set_lateral_mode");
    if (!plan) return bad("dc_fspb_set_lateral_mode: NULL argument");
    if (mode != DC_LATERAL_ISO && mode != DC_LATERAL_AXIS && mode != DC_LATERAL_MLP)
        return bad("dc_fspb_set_lateral_mode: unknown mode");
    if (mode == DC_LATERAL_MLP && !plan->mlp_ready)
        return bad("dc_fspb_set_lateral_mode: the network form needs dc_fspb_set_surrogate first");
    plan->lateral_mode = mode;
    ++plan->layout_gen;
    if (plan->coeffs.density_correction && mode != DC_LATERAL_ISO) DC_CUDA(launch_lateral(plan));
    if (plan->sp_ready) plan->spmm_invalidate();   // matrix values depend on the form
    return DC_OK;
}

dc_status dc_fspb_set_precision(dc_plan* plan, int32_t precision)
{
    if (!plan) return bad("dc_fspb_set_precision: NULL argument");
    if (precision != DC_PRECISION_FP32 && precision != DC_PRECISION_BF16)
        return bad("dc_fspb_set_precision: unknown precision");
    plan->precision = precision;
    ++plan->layout_gen;   // a captured batch graph picks its kernel by it
    return DC_OK;
}

dc_status dc_fspb_lateral_fallbacks(dc_plan* plan, int64_t* n)
{
    if (!plan || !n) return bad("dc_fspb_lateral_fallbacks: NULL argument");
    int32_t h = 0;
    DC_CUDA(cudaMemcpyAsync(&h, plan->d_nfall, sizeof(int32_t), cudaMemcpyDeviceToHost, plan->stream));
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    *n = h;
    return DC_OK;
}

dc_status dc_fspb_stencils(dc_plan* plan, const int32_t* vox, const int32_t* beam, int32_t n, float* X, float* T,
                           uint32_t flags)
{
    DC_NVTX("dc_fspb_stencils");
    if (!plan || !vox || !beam || !X || !T) return bad("dc_fspb_stencils: NULL argument");
    if (n < 0) return bad("dc_fspb_stencils: n < 0");
    if (n == 0) return DC_OK;
    if (flags & DC_DEVICE_PTRS) {
        DC_CUDA(launch_stencils(plan, vox, beam, n, X, T));
        return DC_OK;
    }
    for (int s = 0; s < n; ++s)
        if (vox[s] < 0 || vox[s] >= plan->V || beam[s] < 0 || beam[s] >= plan->n_beams)
            return bad("dc_fspb_stencils: voxel or beam index out of range (sample " + std::to_string(s) + ")");
    int32_t *dv = nullptr, *db = nullptr;
    float *dX = nullptr, *dT = nullptr;
    cudaError_t e = dc::dev_malloc(&dv, n * sizeof(int32_t));
    if (e == cudaSuccess) e = dc::dev_malloc(&db, n * sizeof(int32_t));
    if (e == cudaSuccess) e = dc::dev_malloc(&dX, (size_t)n * 48 * sizeof(float));
    if (e == cudaSuccess) e = dc::dev_malloc(&dT, (size_t)n * 3 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dv, vox, n * sizeof(int32_t), cudaMemcpyHostToDevice, plan->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, beam, n * sizeof(int32_t), cudaMemcpyHostToDevice, plan->stream);
    if (e == cudaSuccess) e = launch_stencils(plan, dv, db, n, dX, dT);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(X, dX, (size_t)n * 48 * sizeof(float), cudaMemcpyDeviceToHost, plan->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T, dT, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost, plan->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
    cudaFree(dv);
    cudaFree(db);
    cudaFree(dX);
    cudaFree(dT);
    if (e != cudaSuccess) return cuda_fail(e, "dc_fspb_stencils");
    return DC_OK;
}

dc_status dc_mlp_create(const float* params, void* cuda_stream, dc_mlp** out)
{
    if (!params || !out) return bad("dc_mlp_create: NULL argument");
    *out = nullptr;
    dc_mlp* m = new (std::nothrow) dc_mlp();
    if (!m) return DC_ENOMEM;
    m->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = dc::dev_malloc(&m->theta, kMlpParams * sizeof(float));
    if (e == cudaSuccess) e = dc::dev_malloc(&m->m1, kMlpParams * sizeof(float));
    if (e == cudaSuccess) e = dc::dev_malloc(&m->m2, kMlpParams * sizeof(float));
    if (e == cudaSuccess) e = dc::dev_malloc(&m->grad, kMlpParams * sizeof(float));
    if (e == cudaSuccess) e = dc::dev_malloc(&m->partial, (size_t)kGradCtas * kMlpParams * sizeof(float));
    if (e == cudaSuccess) e = dc::dev_malloc(&m->loss_part, kGradCtas * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->theta, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m1, 0, kMlpParams * sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m2, 0, kMlpParams * sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        mlp_free(m);
        return cuda_fail(e, "dc_mlp_create");
    }
    *out = m;
    return DC_OK;
}

dc_status dc_mlp_destroy(dc_mlp* m)
{
    if (m) {
        cudaStreamSynchronize(m->stream);
        mlp_free(m);
    }
    return DC_OK;
}

dc_status dc_mlp_get_params(const dc_mlp* m, float* out)
{
    if (!m || !out) return bad("dc_mlp_get_params: NULL argument");
    DC_CUDA(cudaMemcpyAsync(out, m->theta, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    DC_CUDA(cudaStreamSynchronize(m->stream));
    return DC_OK;
}

dc_status dc_mlp_get_state(const dc_mlp* m, float* theta, float* m1, float* m2, int64_t* step)
{
    if (!m || !theta || !m1 || !m2 || !step) return bad("dc_mlp_get_state: NULL argument");
    DC_CUDA(cudaMemcpyAsync(theta, m->theta, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    DC_CUDA(cudaMemcpyAsync(m1, m->m1, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    DC_CUDA(cudaMemcpyAsync(m2, m->m2, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    DC_CUDA(cudaStreamSynchronize(m->stream));
    *step = m->step;
    return DC_OK;
}

dc_status dc_mlp_set_state(dc_mlp* m, const float* theta, const float* m1, const float* m2, int64_t step)
{
    if (!m || !theta || !m1 || !m2) return bad("dc_mlp_set_state: NULL argument");
    if (step < 0) return bad("dc_mlp_set_state: step < 0");
    for (int q = 0; q < kMlpParams; ++q)
        if (!isfinite(theta[q]) || !isfinite(m1[q]) || !(m2[q] >= 0.f) || !isfinite(m2[q]))
            return bad("dc_mlp_set_state: non-finite parameter or moment, or a negative second moment");
    DC_CUDA(cudaStreamSynchronize(m->stream));
    DC_CUDA(cudaMemcpyAsync(m->theta, theta, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    DC_CUDA(cudaMemcpyAsync(m->m1, m1, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    DC_CUDA(cudaMemcpyAsync(m->m2, m2, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    DC_CUDA(cudaStreamSynchronize(m->stream));
    m->step = (int)step;
    return DC_OK;
}

// Device copies of the samples (host inputs are uploaded into the trainer's buffers).
static dc_status stage(dc_mlp* m, const float*& X, const float*& T, int n, uint32_t flags)
{
    if (flags & DC_DEVICE_PTRS) return DC_OK;
    if ((size_t)n > m->cap) {
        if (m->dX) cudaFree(m->dX);
        if (m->dT) cudaFree(m->dT);
        m->dX = m->dT = nullptr;
        m->cap = 0;
        DC_CUDA(dc::dev_malloc(&m->dX, (size_t)n * 48 * sizeof(float)));
        DC_CUDA(dc::dev_malloc(&m->dT, (size_t)n * 3 * sizeof(float)));
        m->cap = n;
    }
    DC_CUDA(cudaMemcpyAsync(m->dX, X, (size_t)n * 48 * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    DC_CUDA(cudaMemcpyAsync(m->dT, T, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    X = m->dX;
    T = m->dT;
    return DC_OK;
}

// Per-CTA partial gradients of n samples in the trainer's precision.
static cudaError_t grad_kernel(dc_mlp* m, int nctas, const float* X, const float* T, int n)
{
    if (m->precision == DC_PRECISION_BF16)
        return launch_mlp_grad_bf16(m->stream, nctas, m->theta, X, T, n, m->partial, m->loss_part);
    return launch_mlp_grad(m->stream, nctas, m->theta, X, T, n, m->partial, m->loss_part);
}

dc_status dc_mlp_set_precision(dc_mlp* m, int32_t precision)
{
    if (!m) return bad("dc_mlp_set_precision: NULL argument");
    if (precision != DC_PRECISION_FP32 && precision != DC_PRECISION_BF16)
        return bad("dc_mlp_set_precision: unknown precision");
    m->precision = precision;
    return DC_OK;
}

// Loss and gradient (FP32) of the current parameters on n samples, summed in a fixed order.
static dc_status grad_pass(dc_mlp* m, const float* X, const float* T, int n, float* loss_host)
{
    const int tiles = (n + 63) / 64;
    const int nctas = tiles < kGradCtas ? tiles : kGradCtas;
    DC_CUDA(grad_kernel(m, nctas, X, T, n));
    DC_CUDA(launch_mlp_adam(m->stream, m->partial, nctas, m->theta, m->m1, m->m2, m->grad, 0.f, 0.9f, 0.999f, 1e-8f, 1));
    if (loss_host) {
        std::vector<float> lp(nctas);
        DC_CUDA(cudaMemcpyAsync(lp.data(), m->loss_part, nctas * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        DC_CUDA(cudaStreamSynchronize(m->stream));
        double s = 0.0;
        for (float x : lp) s += x;
        *loss_host = (float)(s / (3.0 * n));
    }
    return DC_OK;
}

dc_status dc_mlp_gradient(dc_mlp* m, const float* X, const float* T, int32_t n, float* grad, float* loss, uint32_t flags)
{
    DC_NVTX("dc_mlp_gradient");
    if (!m || !X || !T || !grad) return bad("dc_mlp_gradient: NULL argument");
    if (n < 1) return bad("dc_mlp_gradient: n < 1");
    dc_status s = stage(m, X, T, n, flags);
    if (s != DC_OK) return s;
    s = grad_pass(m, X, T, n, loss);
    if (s != DC_OK) return s;
    DC_CUDA(cudaMemcpyAsync(grad, m->grad, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    DC_CUDA(cudaStreamSynchronize(m->stream));
    return DC_OK;
}

dc_status dc_mlp_train(dc_mlp* m, const float* X, const float* T, int32_t n, int32_t batch, int32_t epochs, float lr,
                       float* loss, uint32_t flags)
{
    DC_NVTX("dc_mlp_train");
    if (!m || !X || !T) return bad("dc_mlp_train: NULL argument");
    if (n < 1 || batch < 1 || epochs < 0 || !(lr > 0)) return bad("dc_mlp_train: bad n, batch, epochs or lr");
    dc_status s = stage(m, X, T, n, flags);
    if (s != DC_OK) return s;
    // whole batches in the given (pre-shuffled) order: a gradient and an Adam
    // launch per step, on stream `st`
    auto steps = [&](cudaStream_t st) -> cudaError_t {
        const int tiles = (batch + 63) / 64;
        const int nctas = tiles < kGradCtas ? tiles : kGradCtas;
        for (int ep = 0; ep < epochs; ++ep)
            for (int b0 = 0; b0 + batch <= n; b0 += batch) {
                const cudaStream_t own = m->stream;
                m->stream = st;
                cudaError_t e = grad_kernel(m, nctas, X + (size_t)b0 * 48, T + (size_t)b0 * 3, batch);
                m->stream = own;
                if (e != cudaSuccess) return e;
                ++m->step;
                e = launch_mlp_adam(st, m->partial, nctas, m->theta, m->m1, m->m2, nullptr, lr, 0.9f, 0.999f, 1e-8f,
                                    m->step);
                if (e != cudaSuccess) return e;
            }
        return cudaSuccess;
    };
    const int64_t n_steps = (int64_t)epochs * (n / batch);
    if (n_steps < 8) {
        DC_CUDA(steps(m->stream));
    } else {
        // many small launches: captured once as a CUDA graph (on a stream of
        // its own, ordered after and before the trainer's stream), so that
        // they run back to back without a host launch in between
        cudaStream_t cs = nullptr;
        cudaEvent_t ev = nullptr;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        const int64_t step0 = m->step;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, m->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t ec = steps(cs);
            const cudaError_t ee = cudaStreamEndCapture(cs, &g);
            e = ec != cudaSuccess ? ec : ee;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        bool launched = false;
        if (e == cudaSuccess) {
            e = cudaGraphLaunch(ge, cs);
            launched = e == cudaSuccess;
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m->stream, ev, 0);
        if (!launched) m->step = step0;   // the captured steps never ran
        if (ge) cudaGraphExecDestroy(ge);         // freed when the replay ends
        if (g) cudaGraphDestroy(g);
        if (ev) cudaEventDestroy(ev);
        if (cs) cudaStreamDestroy(cs);
        if (e != cudaSuccess) return cuda_fail(e, "dc_mlp_train");
    }
    if (loss) return grad_pass(m, X, T, n, loss);
    DC_CUDA(cudaStreamSynchronize(m->stream));
    return DC_OK;
}

dc_status dc_mlp_predict(const float* params, const float* X, int32_t n, float* Y, uint32_t flags, void* cuda_stream)
{
    DC_NVTX("dc_mlp_predict");
    if (!params || !X || !Y) return bad("dc_mlp_predict: NULL argument");
    if (n < 1) return bad("dc_mlp_predict: n < 1");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    std::vector<uint2> frag;
    std::vector<float> bias;
    mlp_pack(params, frag, bias);
    uint2* df = nullptr;
    float *db = nullptr, *dX = nullptr, *dY = nullptr;
    const bool dev = flags & DC_DEVICE_PTRS;
    cudaError_t e = dc::dev_malloc(&df, frag.size() * sizeof(uint2));
    if (e == cudaSuccess) e = dc::dev_malloc(&db, bias.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(df, frag.data(), frag.size() * sizeof(uint2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, bias.data(), bias.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (!dev) {
        if (e == cudaSuccess) e = dc::dev_malloc(&dX, (size_t)n * 48 * sizeof(float));
        if (e == cudaSuccess) e = dc::dev_malloc(&dY, (size_t)n * 3 * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpyAsync(dX, X, (size_t)n * 48 * sizeof(float), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = launch_mlp_predict_bf16(st, dev ? X : dX, n, df, db, dev ? Y : dY);
    if (!dev && e == cudaSuccess) e = cudaMemcpyAsync(Y, dY, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(df);
    cudaFree(db);
    if (dX) cudaFree(dX);
    if (dY) cudaFree(dY);
    if (e != cudaSuccess) return cuda_fail(e, "dc_mlp_predict");
    return DC_OK;
}

}  // extern "C"
