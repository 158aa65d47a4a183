// Multi-plan batch: the eq. (1) dose of several plans (uneven grids and beam
// counts) as one persistent pair-kernel launch over the work units of all
// plans, replayed from a CUDA graph.  With DC_BATCH_DENSITY the graph also
// holds each plan's density-dependent steps (Algorithm A1 steps 1-6, the
// beam's-eye-view binning and the lateral factors), one branch per plan, so a
// replay recomputes whole plans from their resident densities.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "dc_internal.cuh"

using namespace dc;

struct dc_batch {
    int device = 0;
    int n = 0;
    std::vector<dc_plan*> plans;        // caller order
    std::vector<int> order;             // position in the unit range -> caller index (costliest first)
    cudaStream_t stream = nullptr;      // runs are launched here
    cudaStream_t cap = nullptr;         // capture origin
    std::vector<cudaStream_t> side;     // per-plan branches of the density graph
    cudaEvent_t fork = nullptr, done = nullptr;
    std::vector<cudaEvent_t> join;      // branch ends inside the captured graph
    std::vector<cudaEvent_t> pre;       // plans' pending work, before a replay
    std::vector<DoseArgs> h_args;       // [n], in unit-range order
    DoseArgs* d_args = nullptr;         // device copy
    int64_t* d_prefix = nullptr;        // [groups][n + 1] unit prefix per plan group (device-computed)
    int64_t* d_vpre = nullptr;          // [n + 1] voxel prefix
    unsigned int* d_counter = nullptr;
    std::vector<float*> d_fluence, d_dose;   // caller order, owned by the batch
    int64_t v_total = 0;
    bool shared_water = false;          // all plans use identical water tables
    int kvariant = 0;                   // 0, 1: register budget of the batch pair kernel; kBatchPerPlan (dc_fspb_batch_autotune)
    cudaGraphExec_t exec[2] = {nullptr, nullptr};   // [0] dose, [1] density steps + dose
    int kernels[2] = {0, 0};                        // kernel nodes per replay
    std::vector<uint64_t> gen;                      // plans' layout_gen when args were written

    void drop_graphs()
    {
        for (auto& e : exec)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
    }
    ~dc_batch()
    {
        drop_graphs();
        for (float* b : d_fluence)
            if (b) cudaFree(b);
        for (float* b : d_dose)
            if (b) cudaFree(b);
        void* bufs[] = {d_args, d_prefix, d_vpre, d_counter};
        for (void* b : bufs)
            if (b) cudaFree(b);
        for (cudaStream_t s : side)
            if (s) cudaStreamDestroy(s);
        if (cap) cudaStreamDestroy(cap);
        for (cudaEvent_t e : join)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : pre)
            if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (done) cudaEventDestroy(done);
    }
};

namespace {

dc_status bad(const std::string& msg)
{
    set_error(msg);
    return DC_EINVAL;
}

uint64_t launches_now()
{
    uint64_t n = 0;
    dc_fspb_launch_count(&n);
    return n;
}

// Writes the per-plan kernel arguments (in unit-range order) when a plan's
// buffers or launch parameters changed since they were last written; stale
// graphs are dropped.
dc_status refresh_args(dc_batch* bt)
{
    bool stale = bt->gen.empty();
    for (int i = 0; i < bt->n && !stale; ++i) stale = bt->gen[i] != bt->plans[i]->layout_gen;
    if (!stale) return DC_OK;
    bt->drop_graphs();
    std::vector<DoseArgs>& args = bt->h_args;
    args.resize(bt->n);
    for (int j = 0; j < bt->n; ++j) {
        const int i = bt->order[j];
        args[j] = dose_args(bt->plans[i], bt->d_fluence[i], bt->d_dose[i]);
    }
    DC_CUDA(cudaMemcpyAsync(bt->d_args, args.data(), sizeof(DoseArgs) * bt->n, cudaMemcpyHostToDevice, bt->cap));
    DC_CUDA(cudaStreamSynchronize(bt->cap));
    bt->gen.resize(bt->n);
    for (int i = 0; i < bt->n; ++i) bt->gen[i] = bt->plans[i]->layout_gen;
    return DC_OK;
}

// Enqueues the work of one replay on the capture stream (while it is captured).
cudaError_t enqueue(dc_batch* bt, bool density)
{
    cudaError_t e = cudaSuccess;
    if (density) {
        e = cudaEventRecord(bt->fork, bt->cap);
        if (e != cudaSuccess) return e;
        for (int j = 0; j < bt->n; ++j) {
            dc_plan* p = bt->plans[bt->order[j]];
            cudaStream_t br = bt->side[j];
            e = cudaStreamWaitEvent(br, bt->fork, 0);
            if (e != cudaSuccess) return e;
            // the plan's launchers enqueue on p->stream: point it at the branch
            cudaStream_t own = p->stream;
            p->stream = br;
            e = launch_smooth(p, p->coeffs.smooth_sigma);
            if (e == cudaSuccess) e = launch_factors(p);
            if (e == cudaSuccess) e = launch_beamlets(p);
            if (e == cudaSuccess) e = launch_binning(p);
            if (e == cudaSuccess && p->coeffs.density_correction && p->lateral_mode != DC_LATERAL_ISO)
                e = launch_lateral(p);
            if (e == cudaSuccess) e = cudaMemsetAsync(p->d_part, 0, sizeof(float) * (size_t)p->n_beams * p->V, br);
            p->stream = own;
            if (e != cudaSuccess) return e;
            e = cudaEventRecord(bt->join[j], br);
            if (e != cudaSuccess) return e;
            e = cudaStreamWaitEvent(bt->cap, bt->join[j], 0);
            if (e != cudaSuccess) return e;
        }
    } else if (bt->kvariant != kBatchPerPlan) {
        for (int j = 0; j < bt->n; ++j) {
            dc_plan* p = bt->plans[bt->order[j]];
            e = cudaMemsetAsync(p->d_part, 0, sizeof(float) * (size_t)p->n_beams * p->V, bt->cap);
            if (e != cudaSuccess) return e;
        }
    }
    if (bt->kvariant == kBatchPerPlan) {
        // each plan's own dose launch (its pair kernel specialised for that
        // plan alone, then its beam sums), one after another in the graph
        for (int j = 0; j < bt->n; ++j) {
            const int i = bt->order[j];
            dc_plan* p = bt->plans[i];
            cudaStream_t own = p->stream;
            p->stream = bt->cap;
            e = launch_dose(p, bt->d_fluence[i], 1, p->B, bt->d_dose[i], p->V);
            p->stream = own;
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    return launch_batch(bt->cap, bt->h_args.data(), bt->d_args, bt->n, bt->d_vpre, bt->v_total, bt->d_prefix,
                        bt->d_counter, bt->device, bt->kvariant, bt->shared_water);
}

dc_status capture(dc_batch* bt, int variant)
{
    const uint64_t before = launches_now();
    DC_CUDA(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
    const cudaError_t e = enqueue(bt, variant == 1);
    cudaGraph_t g = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(bt->cap, &g);
    // kernels enqueued during capture ran no work: take them off the counter
    const uint64_t captured = launches_now() - before;
    count_launches(-(int)captured);
    if (e != cudaSuccess || e_end != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e != cudaSuccess ? e : e_end, "batch graph capture");
    }
    const cudaError_t e_inst = cudaGraphInstantiate(&bt->exec[variant], g, 0);
    cudaGraphDestroy(g);
    if (e_inst != cudaSuccess) {
        bt->exec[variant] = nullptr;
        return cuda_fail(e_inst, "cudaGraphInstantiate");
    }
    bt->kernels[variant] = (int)captured;
    return DC_OK;
}

// Orders the batch stream after each plan's pending work, replays the graph,
// and orders each plan's stream after the replay.
dc_status run(dc_batch* bt, uint32_t flags)
{
    const int variant = (flags & DC_BATCH_DENSITY) ? 1 : 0;
    dc_status s = refresh_args(bt);
    if (s != DC_OK) return s;
    if (!bt->exec[variant]) {
        s = capture(bt, variant);
        if (s != DC_OK) return s;
    }
    if (variant == 1)
        for (dc_plan* p : bt->plans) {
            // the voxel lists are rebuilt: the matrix pattern and SpMM tiles follow them
            DC_CUDA(cudaStreamSynchronize(p->stream));
            p->pairs = -1;
            p->counts_fresh = false;
            if (p->sp_ready) p->spmm_invalidate();
        }
    for (int i = 0; i < bt->n; ++i) {
        DC_CUDA(cudaEventRecord(bt->pre[i], bt->plans[i]->stream));
        DC_CUDA(cudaStreamWaitEvent(bt->stream, bt->pre[i], 0));
    }
    DC_CUDA(cudaGraphLaunch(bt->exec[variant], bt->stream));
    count_launches(bt->kernels[variant]);
    DC_CUDA(cudaEventRecord(bt->done, bt->stream));
    for (dc_plan* p : bt->plans) DC_CUDA(cudaStreamWaitEvent(p->stream, bt->done, 0));
    return DC_OK;
}

}  // namespace

extern "C" {

dc_status dc_fspb_batch_create(dc_plan* const* plans, int32_t n, void* cuda_stream, dc_batch** out)
{
    DC_NVTX("dc_fspb_batch_create");
    if (!out) return bad("dc_fspb_batch_create: out is NULL");
    *out = nullptr;
    if (!plans) return bad("dc_fspb_batch_create: plans is NULL");
    if (n < 1 || n > batch_max_plans())
        return bad("dc_fspb_batch_create: n must be in [1, " + std::to_string(batch_max_plans()) + "]");
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return bad("dc_fspb_batch_create: plan " + std::to_string(i) + " is NULL");
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return bad("dc_fspb_batch_create: a plan appears twice");
        if (plans[i]->device != plans[0]->device)
            return bad("dc_fspb_batch_create: plans on different devices");
    }
    int cur = -1;
    DC_CUDA(cudaGetDevice(&cur));
    if (cur != plans[0]->device) return bad("dc_fspb_batch_create: the plans' device is not the current device");

    dc_batch* bt = new (std::nothrow) dc_batch();
    if (!bt) {
        set_error("dc_fspb_batch_create: host allocation failed");
        return DC_ENOMEM;
    }
    auto fail = [&](dc_status s) {
        delete bt;
        return s;
    };
    bt->device = plans[0]->device;
    bt->n = n;
    bt->plans.assign(plans, plans + n);
    bt->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    // costliest plans first, so the end of the unit range holds the small units
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i)
        cost[i] = plans[i]->pairs >= 0 ? (double)plans[i]->pairs : (double)plans[i]->B * (double)plans[i]->V;
    bt->order.resize(n);
    for (int i = 0; i < n; ++i) bt->order[i] = i;
    std::stable_sort(bt->order.begin(), bt->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

    cudaError_t e = cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreateWithFlags"));
    bt->side.assign(n, nullptr);
    bt->join.assign(n, nullptr);
    bt->pre.assign(n, nullptr);
    for (int j = 0; j < n; ++j) {
        e = cudaStreamCreateWithFlags(&bt->side[j], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->join[j], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->pre[j], cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(cuda_fail(e, "batch streams"));
    }
    e = cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->done, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(cuda_fail(e, "batch events"));

    bt->d_fluence.assign(n, nullptr);
    bt->d_dose.assign(n, nullptr);
    std::vector<int64_t> vpre(n + 1, 0);
    for (int j = 0; j < n; ++j) vpre[j + 1] = vpre[j] + plans[bt->order[j]]->V;
    bt->v_total = vpre[n];
    for (int i = 0; i < n; ++i) {
        e = dc::dev_malloc(&bt->d_fluence[i], sizeof(float) * (size_t)plans[i]->B);
        if (e == cudaSuccess) e = dc::dev_malloc(&bt->d_dose[i], sizeof(float) * (size_t)plans[i]->V);
        if (e == cudaSuccess) e = cudaMemset(bt->d_fluence[i], 0, sizeof(float) * (size_t)plans[i]->B);
        if (e != cudaSuccess) return fail(cuda_fail(e, "batch buffers"));
    }
    e = dc::dev_malloc(&bt->d_args, sizeof(DoseArgs) * n);
    if (e == cudaSuccess) e = dc::dev_malloc(&bt->d_prefix, sizeof(int64_t) * batch_groups() * (n + 1));
    if (e == cudaSuccess) e = dc::dev_malloc(&bt->d_vpre, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess) e = dc::dev_malloc(&bt->d_counter, sizeof(unsigned int) * batch_groups());
    if (e == cudaSuccess) e = cudaMemcpy(bt->d_vpre, vpre.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_fail(e, "batch set-up"));
    // one set of water tables for all plans (the usual case: one beam model)?
    {
        const dc_plan* p0 = plans[0];
        bool same = true;
        for (int i = 1; i < n && same; ++i)
            same = plans[i]->coeffs.w_n == p0->coeffs.w_n && plans[i]->coeffs.w_dt == p0->coeffs.w_dt;
        if (same && n > 1) {
            const size_t bytes = 2 * sizeof(float4) * (size_t)p0->coeffs.w_n;
            std::vector<unsigned char> w0(bytes), wi(bytes);
            e = cudaMemcpy(w0.data(), p0->d_water, bytes, cudaMemcpyDeviceToHost);
            for (int i = 1; i < n && same && e == cudaSuccess; ++i) {
                e = cudaMemcpy(wi.data(), plans[i]->d_water, bytes, cudaMemcpyDeviceToHost);
                same = e == cudaSuccess && memcmp(w0.data(), wi.data(), bytes) == 0;
            }
            if (e != cudaSuccess) return fail(cuda_fail(e, "batch water tables"));
        }
        bt->shared_water = same;
    }
    for (dc_plan* p : bt->plans) {
        e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamSynchronize"));
    }
    dc_status s = refresh_args(bt);
    if (s != DC_OK) return fail(s);
    *out = bt;
    return DC_OK;
}

dc_status dc_fspb_batch_destroy(dc_batch* batch)
{
    if (!batch) return DC_OK;
    cudaStreamSynchronize(batch->stream);
    cudaStreamSynchronize(batch->cap);
    delete batch;
    return DC_OK;
}

dc_status dc_fspb_batch_buffers(dc_batch* batch, int32_t i, float** fluence, float** dose)
{
    if (!batch) return bad("dc_fspb_batch_buffers: NULL batch");
    if (i < 0 || i >= batch->n) return bad("dc_fspb_batch_buffers: plan index out of range");
    if (fluence) *fluence = batch->d_fluence[i];
    if (dose) *dose = batch->d_dose[i];
    return DC_OK;
}

dc_status dc_fspb_batch_run(dc_batch* batch, uint32_t flags)
{
    DC_NVTX("dc_fspb_batch_run");
    if (!batch) return bad("dc_fspb_batch_run: NULL batch");
    if (flags & ~(uint32_t)DC_BATCH_DENSITY) return bad("dc_fspb_batch_run: unknown flags");
    return run(batch, flags);
}

dc_status dc_fspb_batch_dose(dc_batch* batch, const float* const* fluence, float* const* dose, uint32_t flags)
{
    DC_NVTX("dc_fspb_batch_dose");
    if (!batch || !fluence || !dose) return bad("dc_fspb_batch_dose: NULL argument");
    if (flags & ~(uint32_t)(DC_DEVICE_PTRS | DC_BATCH_DENSITY)) return bad("dc_fspb_batch_dose: unknown flags");
    for (int i = 0; i < batch->n; ++i)
        if (!fluence[i] || !dose[i]) return bad("dc_fspb_batch_dose: NULL buffer of plan " + std::to_string(i));
    const cudaMemcpyKind kin = (flags & DC_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = (flags & DC_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int i = 0; i < batch->n; ++i)
        DC_CUDA(cudaMemcpyAsync(batch->d_fluence[i], fluence[i], sizeof(float) * (size_t)batch->plans[i]->B, kin,
                                batch->stream));
    dc_status s = run(batch, flags & DC_BATCH_DENSITY);
    if (s != DC_OK) return s;
    for (int i = 0; i < batch->n; ++i)
        DC_CUDA(cudaMemcpyAsync(dose[i], batch->d_dose[i], sizeof(float) * (size_t)batch->plans[i]->V, kout,
                                batch->stream));
    DC_CUDA(cudaStreamSynchronize(batch->stream));
    return DC_OK;
}

dc_status dc_fspb_batch_synchronize(dc_batch* batch)
{
    if (!batch) return bad("dc_fspb_batch_synchronize: NULL batch");
    DC_CUDA(cudaStreamSynchronize(batch->stream));
    return DC_OK;
}

dc_status dc_fspb_batch_autotune(dc_batch* batch, int32_t* variant, float* ms)
{
    DC_NVTX("dc_fspb_batch_autotune");
    if (!batch) return bad("dc_fspb_batch_autotune: NULL batch");
    float best_ms = 0.f;
    int best = -1;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    DC_CUDA(cudaEventCreate(&t0));
    cudaError_t e = cudaEventCreate(&t1);
    if (e != cudaSuccess) {
        cudaEventDestroy(t0);
        return cuda_fail(e, "cudaEventCreate");
    }
    dc_status s = DC_OK;
    for (int v = 0; v <= kBatchPerPlan && s == DC_OK; ++v) {
        batch->kvariant = v;
        batch->drop_graphs();
        s = run(batch, 0);   // captures, and warms up
        float sum = 0.f;
        for (int r = 0; r < 2 && s == DC_OK; ++r) {
            e = cudaEventRecord(t0, batch->stream);
            if (e == cudaSuccess) s = run(batch, 0);
            if (s == DC_OK && e == cudaSuccess) e = cudaEventRecord(t1, batch->stream);
            if (s == DC_OK && e == cudaSuccess) e = cudaEventSynchronize(t1);
            float t = 0.f;
            if (s == DC_OK && e == cudaSuccess) e = cudaEventElapsedTime(&t, t0, t1);
            if (e != cudaSuccess && s == DC_OK) s = cuda_fail(e, "dc_fspb_batch_autotune timing");
            sum += t;
        }
        if (s == DC_OK && (best < 0 || sum < best_ms)) {
            best = v;
            best_ms = sum;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (s != DC_OK) return s;
    batch->kvariant = best;
    batch->drop_graphs();
    if (variant) *variant = best;
    if (ms) *ms = best_ms / 2;
    return DC_OK;
}

dc_status dc_fspb_batch_set_variant(dc_batch* batch, int32_t variant)
{
    if (!batch) return bad("dc_fspb_batch_set_variant: NULL batch");
    if (variant < 0 || variant > kBatchPerPlan) return bad("dc_fspb_batch_set_variant: variant must be 0, 1 or 2");
    DC_CUDA(cudaStreamSynchronize(batch->stream));
    batch->kvariant = variant;
    batch->drop_graphs();
    return DC_OK;
}

dc_status dc_fspb_batch_kernels(const dc_batch* batch, uint32_t flags, int32_t* kernels)
{
    if (!batch || !kernels) return bad("dc_fspb_batch_kernels: NULL argument");
    const int variant = (flags & DC_BATCH_DENSITY) ? 1 : 0;
    *kernels = batch->exec[variant] ? batch->kernels[variant] : 0;
    return DC_OK;
}

}  // extern "C"
