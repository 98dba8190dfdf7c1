// lll_batch.cpp -- many independent term structures in one persistent launch
// (C ABI lll_batch_*).
//
// Each instance is an ordinary model context (lll_init builds its FP64 tables
// on the GPU).  A simulation of the batch is one launch of batch_kernel: the
// tiles of every instance are cut into work items (runs of consecutive tiles
// of one instance) of at most 1/16 of a resident block's share of the cost,
// and the blocks claim the items in order of decreasing cost from a counter,
// so uneven instances (N from 8 to 80, path budgets from 2^12 to 2^18) keep
// every SM busy to the end whatever the cost model misses.  Every item writes
// its own partial sums; a second kernel adds the partials of each instance in
// tile order, so results are deterministic.  The launch sequence (descriptor
// upload, counter reset, the two kernels) can be captured once in a CUDA
// graph and replayed.  Each scheme (full, Picard) keeps its own launch shape
// (threads, blocks per SM, chunk rows, one or two paths per thread), schedule
// and graph, so alternating schemes rebuilds nothing.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lll.h"
#include "lll_ctx.h"
#include "lll_internal.h"

namespace lll {
int batch_finalize(const double *partials, const size_t *seg_off, const int *inst_seg_ptr,
                   const int *inst_segs, const size_t *out_off, int n_inst, const int *out_count,
                   double *sums, cudaStream_t st);
}

using namespace lll;

namespace {

// Launch shape of one scheme.
struct Shape {
    int threads = 128, blocks_per_sm = 0, chunk_rows = 0, R = 1;
};

// Device schedule of one scheme (built by its first simulation).
struct Sched {
    int *d_item_inst = nullptr, *d_next = nullptr, *d_inst_seg_ptr = nullptr, *d_inst_segs = nullptr;
    uint2 *d_item_tiles = nullptr;
    size_t *d_seg_off = nullptr;
    double *d_partials = nullptr;
    float *d_state = nullptr;
    int grid = 0, n_items = 0, CH = 0, R = 1, threads = 128;
    size_t smem = 0;
    bool built = false;
    cudaGraphExec_t graph = nullptr;
};

}  // namespace

struct lll_batch {
    std::vector<lll_ctx *> inst;
    std::vector<uint64_t> paths;
    cudaStream_t stream = nullptr;
    int sm_count = 0, QP = 0, n_max = 0, ns_max = 0;
    Shape shape[2]; // by scheme: LLL_FULL, LLL_PICARD
    Sched sched[2];
    PathArgs *d_desc = nullptr;
    PathArgs *h_desc = nullptr; // pinned: descriptors of the next launch
    // per-instance outputs (independent of the scheme)
    int *d_out_count = nullptr;
    size_t *d_out_off = nullptr;
    double *d_sums = nullptr;
    size_t n_out_total = 0;
    std::vector<size_t> out_off;
    bool simulated = false, use_graph = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::string err;
};

namespace {

int berr(lll_batch *b, int code, const std::string &m)
{
    if (b) b->err = m;
    record_error(nullptr, code, m.c_str());
    return code;
}

void free_sched(Sched &c)
{
    cudaFree(c.d_item_inst); cudaFree(c.d_next); cudaFree(c.d_inst_seg_ptr); cudaFree(c.d_inst_segs);
    cudaFree(c.d_item_tiles); cudaFree(c.d_seg_off); cudaFree(c.d_partials); cudaFree(c.d_state);
    if (c.graph) cudaGraphExecDestroy(c.graph);
    c = Sched();
}

void free_outputs(lll_batch *b)
{
    cudaFree(b->d_out_count); cudaFree(b->d_out_off); cudaFree(b->d_sums); cudaFree(b->d_desc);
    b->d_out_count = nullptr; b->d_out_off = nullptr; b->d_sums = nullptr; b->d_desc = nullptr;
}

template <class T>
cudaError_t upload(T **d, const std::vector<T> &h, cudaStream_t st)
{
    cudaError_t e = cudaMalloc((void **)d, sizeof(T) * std::max<size_t>(h.size(), 1));
    if (e != cudaSuccess) return e;
    if (!h.empty()) e = cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st);
    return e;
}

// The per-instance output layout and the descriptor buffer (once).
int build_outputs(lll_batch *b)
{
    if (b->d_sums) return LLL_OK;
    const int ni = (int)b->inst.size();
    std::vector<int> out_count(ni);
    b->out_off.assign(ni, 0);
    size_t oo = 0;
    for (int q = 0; q < ni; ++q) {
        b->out_off[q] = oo;
        out_count[q] = b->inst[q]->n * b->inst[q]->ns * 2;
        oo += out_count[q];
    }
    b->n_out_total = oo;
    cudaStream_t st = b->stream;
    bool ok = upload(&b->d_out_count, out_count, st) == cudaSuccess && upload(&b->d_out_off, b->out_off, st) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&b->d_desc, sizeof(PathArgs) * ni) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&b->d_sums, sizeof(double) * std::max<size_t>(oo, 1)) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) {
        free_outputs(b);
        return berr(b, LLL_ENOMEM, "batch output buffers");
    }
    return LLL_OK;
}

// Build the schedule of `scheme` for its launch shape (if not built yet).
int build_schedule(lll_batch *b, int scheme)
{
    Sched &c = b->sched[scheme];
    if (c.built) return LLL_OK;
    int rc = build_outputs(b);
    if (rc != LLL_OK) return rc;
    free_sched(c);
    const Shape &sh = b->shape[scheme];
    const int T = sh.threads, R = sh.R;
    if (!batch_kernel_supported(scheme, b->QP, R))
        return berr(b, LLL_EUNSUPPORTED, "no batch kernel for this Q and paths per thread");
    const int CH = sh.chunk_rows > 0 ? std::min(sh.chunk_rows, b->n_max)
                                     : std::min(b->n_max, std::max(1, (48 * 1024) / (2 * (b->QP / 4) * 16)));
    const int nst = scheme == LLL_PICARD ? 2 : 1;
    // smem as for the path kernel, sized for the largest instance
    size_t smem = path_kernel_smem(b->QP, b->n_max, b->ns_max, T, CH);
    if (smem > 227 * 1024) return berr(b, LLL_EUNSUPPORTED, "batch shared memory exceeds 227 KB");
    int occ = 0;
    cudaError_t e = (cudaError_t)batch_kernel_prepare(scheme, b->QP, R, smem, T, &occ);
    if (e != cudaSuccess) return berr(b, LLL_ECUDA, std::string("batch kernel attributes: ") + cudaGetErrorString(e));
    if (occ < 1) return berr(b, LLL_EUNSUPPORTED, "batch kernel does not fit on an SM");
    const int bps = sh.blocks_per_sm > 0 ? std::min(sh.blocks_per_sm, occ) : occ;
    // Work items: runs of consecutive tiles (T R paths each) of one instance,
    // each of at most 1/16 of a block's share of the total cost (one tile at
    // least).  A tile costs the same whether or not it is full (its idle lanes
    // run along): s n (n+1)/2 path-rate-steps per path, plus kStepCost of them
    // for each of the s n steps, for what a step does once whatever the number
    // of live rates (the increment, chunk staging and synchronisation, the
    // maturity payoffs).
    constexpr double kStepCost = 3.0;
    const int ni = (int)b->inst.size();
    const uint64_t TP = (uint64_t)T * R;
    std::vector<double> tile_cost(ni);
    std::vector<uint64_t> ntile(ni);
    double total = 0.0;
    uint64_t ntiles = 0;
    for (int q = 0; q < ni; ++q) {
        const lll_ctx *ic = b->inst[q];
        ntile[q] = (b->paths[q] + TP - 1) / TP;
        if (ntile[q] > 0xffffffffull) return berr(b, LLL_EINVAL, "instance has more than 2^32 tiles");
        tile_cost[q] = (double)TP * ic->s * ic->n * ((ic->n + 1) / 2.0 + kStepCost);
        total += tile_cost[q] * (double)ntile[q];
        ntiles += ntile[q];
    }
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(ntiles, (uint64_t)bps * b->sm_count));
    const double target = total / ((double)grid * 16.0);
    struct Item {
        int q;
        uint32_t t0, t1;
        double cost;
    };
    std::vector<Item> items;
    for (int q = 0; q < ni; ++q) {
        const uint64_t per = std::max<uint64_t>(1, (uint64_t)(target / tile_cost[q]));
        const uint64_t nit = (ntile[q] + per - 1) / per; // items of this instance, balanced sizes
        for (uint64_t k = 0; k < nit; ++k) {
            const uint64_t t0 = ntile[q] * k / nit, t1 = ntile[q] * (k + 1) / nit;
            items.push_back({q, (uint32_t)t0, (uint32_t)t1, tile_cost[q] * (double)(t1 - t0)});
        }
    }
    if (items.size() > 0x7fffffffull) return berr(b, LLL_EINVAL, "too many work items");
    // claiming order: decreasing cost (ties in instance and tile order)
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });
    const int nitems = (int)items.size();
    std::vector<int> item_inst(nitems);
    std::vector<uint2> item_tiles(nitems);
    std::vector<size_t> seg_off(nitems);
    size_t off = 0;
    for (int k = 0; k < nitems; ++k) {
        item_inst[k] = items[k].q;
        item_tiles[k] = make_uint2(items[k].t0, items[k].t1);
        seg_off[k] = off;
        const lll_ctx *ic = b->inst[items[k].q];
        off += (size_t)ic->n * ic->ns * 2;
    }
    // per instance: its items in tile order
    std::vector<int> inst_seg_ptr(ni + 1, 0), inst_segs;
    std::vector<std::vector<int>> lists(ni);
    for (int k = 0; k < nitems; ++k) lists[items[k].q].push_back(k);
    for (int q = 0; q < ni; ++q) {
        std::sort(lists[q].begin(), lists[q].end(), [&](int x, int y) { return items[x].t0 < items[y].t0; });
        inst_seg_ptr[q] = (int)inst_segs.size();
        inst_segs.insert(inst_segs.end(), lists[q].begin(), lists[q].end());
    }
    inst_seg_ptr[ni] = (int)inst_segs.size();
    cudaStream_t st = b->stream;
    bool ok = upload(&c.d_item_inst, item_inst, st) == cudaSuccess && upload(&c.d_item_tiles, item_tiles, st) == cudaSuccess &&
              upload(&c.d_seg_off, seg_off, st) == cudaSuccess && upload(&c.d_inst_seg_ptr, inst_seg_ptr, st) == cudaSuccess &&
              upload(&c.d_inst_segs, inst_segs, st) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&c.d_next, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&c.d_partials, sizeof(double) * std::max<size_t>(off, 1)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&c.d_state, sizeof(float) * (size_t)grid * R * nst * b->n_max * T) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) {
        free_sched(c);
        return berr(b, LLL_ENOMEM, "batch schedule buffers");
    }
    c.grid = grid;
    c.n_items = nitems;
    c.CH = CH;
    c.R = R;
    c.threads = T;
    c.smem = smem;
    c.built = true;
    return LLL_OK;
}

int launch_all(lll_batch *b, int scheme)
{
    const Sched &c = b->sched[scheme];
    BatchArgs a{};
    a.desc = b->d_desc; a.item_inst = c.d_item_inst; a.item_tiles = c.d_item_tiles; a.seg_off = c.d_seg_off;
    a.partials = c.d_partials; a.state = c.d_state; a.next = c.d_next;
    a.n_items = c.n_items; a.n_max = b->n_max; a.ns_max = b->ns_max;
    a.chunk_rows = c.CH;
    cudaStream_t st = b->stream;
    cudaError_t e = cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(PathArgs) * b->inst.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return (int)e;
    e = cudaMemsetAsync(c.d_next, 0, sizeof(int), st);
    if (e != cudaSuccess) return (int)e;
    e = (cudaError_t)launch_batch_kernel(scheme, b->QP, c.R, c.grid, c.threads, c.smem, st, a);
    if (e != cudaSuccess) return (int)e;
    return batch_finalize(c.d_partials, c.d_seg_off, c.d_inst_seg_ptr, c.d_inst_segs, b->d_out_off,
                          (int)b->inst.size(), b->d_out_count, b->d_sums, st);
}

}  // namespace

extern "C" {

int lll_batch_init(lll_batch **out, int n_inst, const lll_instance *inst, void *cuda_stream)
{
    if (!out || n_inst < 1 || !inst) return berr(nullptr, LLL_EINVAL, "need out, n_inst >= 1 and instances");
    *out = nullptr;
    lll_batch *b = new lll_batch();
    b->stream = (cudaStream_t)cuda_stream;
    for (int q = 0; q < n_inst; ++q) {
        const lll_instance &I = inst[q];
        lll_ctx *c = nullptr;
        int rc = lll_init(&c, I.N, I.tenor_delta, I.L0, I.steps_per_period, I.lambda, I.driver, I.nig, I.Q,
                          I.nodes, I.weights, cuda_stream);
        if (rc != LLL_OK && rc != LLL_EDOMAIN) {
            std::string m = std::string("instance ") + std::to_string(q) + ": " + lll_last_error(nullptr);
            lll_batch_destroy(b);
            return berr(nullptr, rc, m);
        }
        b->inst.push_back(c);
        rc = lll_set_strikes(c, I.n_strikes, I.strikes);
        if (rc == LLL_OK && I.paths == 0) rc = LLL_EINVAL;
        if (rc != LLL_OK) {
            std::string m = std::string("instance ") + std::to_string(q) + ": strikes or paths invalid";
            lll_batch_destroy(b);
            return berr(nullptr, LLL_EINVAL, m);
        }
        b->paths.push_back(I.paths);
        if (q == 0) b->QP = c->QP;
        if (c->QP != b->QP || c->driver != LLL_DRIVER_NIG) {
            lll_batch_destroy(b);
            return berr(nullptr, LLL_EUNSUPPORTED, "batched instances must share the NIG driver and padded Q");
        }
        b->n_max = std::max(b->n_max, c->n);
        b->ns_max = std::max(b->ns_max, c->ns);
    }
    b->sm_count = b->inst[0]->sm_count;
    if (cudaMallocHost((void **)&b->h_desc, sizeof(PathArgs) * n_inst) != cudaSuccess ||
        cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess) {
        lll_batch_destroy(b);
        return berr(nullptr, LLL_ENOMEM, "pinned descriptor buffer or events");
    }
    *out = b;
    return LLL_OK;
}

int lll_batch_set_launch(lll_batch *b, int scheme, int threads_per_block, int blocks_per_sm, int chunk_rows,
                         int paths_per_thread)
{
    if (!b) return berr(nullptr, LLL_EINVAL, "batch is NULL");
    if (scheme != -1 && scheme != LLL_FULL && scheme != LLL_PICARD)
        return berr(b, LLL_EINVAL, "scheme must be LLL_FULL, LLL_PICARD or -1 (both)");
    if (threads_per_block != 0 && (threads_per_block < 32 || threads_per_block > kMaxThreads || threads_per_block % 32))
        return berr(b, LLL_EINVAL, "threads_per_block must be a multiple of 32 in [32, 256]");
    if (blocks_per_sm < 0 || chunk_rows < 0) return berr(b, LLL_EINVAL, "negative launch value");
    if (paths_per_thread < 0 || paths_per_thread > 2) return berr(b, LLL_EINVAL, "paths_per_thread must be 0, 1 or 2");
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return berr(b, LLL_ECUDA, "stream synchronize");
    for (int s = 0; s < 2; ++s) {
        if (scheme != -1 && s != scheme) continue;
        Shape &sh = b->shape[s];
        sh.threads = threads_per_block ? threads_per_block : 128;
        sh.blocks_per_sm = blocks_per_sm;
        sh.chunk_rows = chunk_rows;
        sh.R = paths_per_thread ? paths_per_thread : 1;
        free_sched(b->sched[s]);
    }
    return LLL_OK;
}

int lll_batch_use_graph(lll_batch *b, int enable)
{
    if (!b) return berr(nullptr, LLL_EINVAL, "batch is NULL");
    b->use_graph = enable != 0;
    return LLL_OK;
}

int lll_batch_simulate(lll_batch *b, int scheme, uint64_t seed)
{
    if (!b) return berr(nullptr, LLL_EINVAL, "batch is NULL");
    if (scheme != LLL_FULL && scheme != LLL_PICARD)
        return berr(b, LLL_EINVAL, "the batched launch runs the full or the Picard scheme");
    int rc = build_schedule(b, scheme);
    if (rc != LLL_OK) return rc;
    Sched &c = b->sched[scheme];
    // the previous launch may still read the pinned descriptors
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return berr(b, LLL_ECUDA, "stream synchronize");
    for (size_t q = 0; q < b->inst.size(); ++q) {
        LaunchPlan plan;
        lll_ctx *ic = b->inst[q];
        ic->lpp = 1;
        ic->ppt = c.R;
        ic->chunk_rows = c.CH; // the descriptors carry the schedule's chunk rows
        rc = plan_launch(ic, scheme, 0, b->paths[q], seed, &plan);
        if (rc != LLL_OK) return berr(b, rc, std::string("instance plan: ") + lll_last_error(ic));
        plan.args.inst = (uint32_t)q; // Philox counter word 1: instances draw independent streams
        if (ic->d_snap) { // parity snapshots of this instance (lll_batch_set_snapshots)
            plan.args.snap = ic->d_snap;
            plan.args.snap_stride = ic->snap_stride;
            plan.args.snap_pitch = ic->n_snap;
            plan.args.n_snap = std::min<uint64_t>(ic->n_snap, (b->paths[q] + ic->snap_stride - 1) / ic->snap_stride);
        }
        ic->last_snap_paths = plan.args.n_snap;
        b->h_desc[q] = plan.args;
    }
    cudaStream_t st = b->stream;
    cudaError_t e = cudaEventRecord(b->ev[0], st);
    if (e == cudaSuccess) {
        if (b->use_graph) {
            if (!c.graph) {
                cudaGraph_t g = nullptr;
                cudaStream_t cap = nullptr;
                e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaStream_t keep = b->stream;
                    b->stream = cap;
                    const int lr = launch_all(b, scheme);
                    b->stream = keep;
                    e = cudaStreamEndCapture(cap, &g);
                    if (e == cudaSuccess && lr != 0) e = (cudaError_t)lr;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&c.graph, g, 0);
                if (g) cudaGraphDestroy(g);
                if (cap) cudaStreamDestroy(cap);
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(c.graph, st);
        } else {
            e = (cudaError_t)launch_all(b, scheme);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[1], st);
    if (e != cudaSuccess) return berr(b, LLL_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    b->simulated = true;
    for (lll_ctx *ic : b->inst) ic->simulated = ic->d_snap != nullptr; // snapshots readable
    return LLL_OK;
}

int lll_batch_set_snapshots(lll_batch *b, int q, uint64_t count, uint64_t stride)
{
    if (!b) return berr(nullptr, LLL_EINVAL, "batch is NULL");
    if (q < 0 || q >= (int)b->inst.size()) return berr(b, LLL_EINVAL, "bad instance");
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return berr(b, LLL_ECUDA, "stream synchronize");
    const int rc = lll_set_snapshots(b->inst[q], count, stride);
    if (rc != LLL_OK) return berr(b, rc, lll_last_error(b->inst[q]));
    b->inst[q]->simulated = false;
    return LLL_OK;
}

int lll_batch_get_paths(lll_batch *b, int q, uint64_t first, uint64_t count, float *out)
{
    if (!b) return berr(nullptr, LLL_EINVAL, "batch is NULL");
    if (q < 0 || q >= (int)b->inst.size()) return berr(b, LLL_EINVAL, "bad instance");
    if (!b->simulated) return berr(b, LLL_ESTATE, "no batch simulation to read");
    const int rc = lll_get_paths(b->inst[q], first, count, out);
    if (rc != LLL_OK) return berr(b, rc, lll_last_error(b->inst[q]));
    return LLL_OK;
}

int lll_batch_prices(lll_batch *b, int q, double *prices, double *stderr_)
{
    if (!b) return berr(nullptr, LLL_EINVAL, "batch is NULL");
    if (!b->simulated) return berr(b, LLL_ESTATE, "no batch simulation to read");
    if (q < 0 || q >= (int)b->inst.size() || !prices) return berr(b, LLL_EINVAL, "bad instance or output");
    const lll_ctx *c = b->inst[q];
    const size_t cnt = (size_t)c->n * c->ns;
    std::vector<double> buf(2 * cnt);
    if (cudaMemcpyAsync(buf.data(), b->d_sums + b->out_off[q], sizeof(double) * 2 * cnt, cudaMemcpyDeviceToHost,
                        b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return berr(b, LLL_ECUDA, "reading batch sums");
    const double P = (double)b->paths[q];
    for (size_t e = 0; e < cnt; ++e) {
        const double mean = buf[2 * e] / P;
        prices[e] = mean;
        if (stderr_) {
            const double var = std::max(buf[2 * e + 1] / P - mean * mean, 0.0) * P / std::max(P - 1.0, 1.0);
            stderr_[e] = std::sqrt(var / P);
        }
    }
    return LLL_OK;
}

int lll_batch_kernel_ms(lll_batch *b, float *ms)
{
    if (!b || !ms) return berr(b, LLL_EINVAL, "batch or output is NULL");
    if (!b->simulated) return berr(b, LLL_ESTATE, "no batch simulation timed");
    if (cudaEventSynchronize(b->ev[1]) != cudaSuccess || cudaEventElapsedTime(ms, b->ev[0], b->ev[1]) != cudaSuccess)
        return berr(b, LLL_ECUDA, "batch timing");
    return LLL_OK;
}

void lll_batch_destroy(lll_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    free_sched(b->sched[0]);
    free_sched(b->sched[1]);
    free_outputs(b);
    if (b->h_desc) cudaFreeHost(b->h_desc);
    for (auto &e : b->ev)
        if (e) cudaEventDestroy(e);
    for (lll_ctx *c : b->inst) lll_destroy(c);
    delete b;
}

}  // extern "C"
