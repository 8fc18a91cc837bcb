// Ragged batches: host side of fwr_batch_* (include/fwr.h). A batch holds the
// device descriptors of its plans, each frame's plan index, the per-CTA frame
// lists of the schedule and (when a 256^2 plan is present) the slab scratch.
// Running a batch is one kernel launch (fwr_ragged.cu) with no allocation and
// no host synchronisation, so it can be captured in a CUDA graph.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <queue>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/fwr.h"
#include "fwr_internal.h"
#include "fwr_plan.h"

struct fwr_batch {
    int device = 0, n_frames = 0, iters = 0, sms = 0;
    std::vector<fwr_plan*> plans;
    std::vector<int> frame_plan;
    int ctas = 0;
    double cost_ratio = 0;
    int shape = 2;  // warp groups of the 256^2 path (1 or 2)
    size_t smem = 0;
    fwr::RaggedPlan* d_plans = nullptr;
    int* d_frame_plan = nullptr;
    int* d_off = nullptr;
    int* d_order = nullptr;
    float2* d_scratch = nullptr;
};

namespace {

const double kDefaultCostRatio = 9.6;  // measured time of a 256^2 frame over a 128^2 frame (k = 5)

void free_batch(fwr_batch* b) {
    cudaFree(b->d_plans);
    cudaFree(b->d_frame_plan);
    cudaFree(b->d_off);
    cudaFree(b->d_order);
    cudaFree(b->d_scratch);
    delete b;
}

}  // namespace

extern "C" {

fwr_status fwr_schedule_lpt(const double* costs, int n, int ctas, int* cta_off, int* order) {
    if (n < 0 || ctas < 1 || (n > 0 && (!costs || !order)) || !cta_off) return FWR_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!(costs[i] >= 0.0) || !std::isfinite(costs[i])) return FWR_ERR_ARG;
    // longest processing time first: the costliest frame goes to the least
    // loaded CTA (ties: lower frame index first, lower CTA index first)
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return costs[a] > costs[b]; });
    typedef std::pair<double, int> Load;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int c = 0; c < ctas; ++c) heap.push(Load(0.0, c));
    std::vector<std::vector<int>> lists(ctas);
    for (int i : idx) {
        Load l = heap.top();
        heap.pop();
        lists[l.second].push_back(i);
        heap.push(Load(l.first + costs[i], l.second));
    }
    int pos = 0;
    for (int c = 0; c < ctas; ++c) {
        cta_off[c] = pos;
        for (int f : lists[c]) order[pos++] = f;
    }
    cta_off[ctas] = pos;
    return FWR_OK;
}

fwr_status fwr_batch_create(fwr_batch** out, fwr_plan* const* plans, int n_plans, const int* frame_plan,
                            int n_frames, int iters) {
    if (!out) return FWR_ERR_ARG;
    *out = nullptr;
    if (!plans || n_plans < 1 || n_frames < 0 || (n_frames > 0 && !frame_plan) || iters < 0 || iters > 64)
        return FWR_ERR_ARG;
    size_t smem = 0;
    bool need_scratch = false;
    int device = -1;
    for (int i = 0; i < n_plans; ++i) {
        const fwr_plan* p = plans[i];
        if (!p) return FWR_ERR_ARG;
        if (device >= 0 && p->device != device) return FWR_ERR_ARG;
        device = p->device;
        const size_t b = fwr::ragged_smem_bytes(p->N, p->n);
        if (b == 0 || b > size_t(227) * 1024) {
            fwr::set_last_error("fwr_batch_create: ragged batches take 128x128 and 256x256 plans "
                                "(128x128 with at most 85 lenslets across)");
            return FWR_ERR_UNSUPPORTED;
        }
        smem = std::max(smem, b);
        need_scratch |= p->N == 256;
    }
    for (int f = 0; f < n_frames; ++f)
        if (frame_plan[f] < 0 || frame_plan[f] >= n_plans) return FWR_ERR_ARG;

    fwr_batch* b = new (std::nothrow) fwr_batch();
    if (!b) return FWR_ERR_CUDA;
    b->device = device;
    b->n_frames = n_frames;
    b->iters = iters;
    b->plans.assign(plans, plans + n_plans);
    b->frame_plan.assign(frame_plan, frame_plan + n_frames);
    b->smem = smem;
    cudaError_t e;
    int prev = 0;
    cudaGetDevice(&prev);
    if ((e = cudaSetDevice(device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) {
        free_batch(b);
        cudaSetDevice(prev);
        return fwr::cuda_fail(e, "fwr_batch_create");
    }
    std::vector<fwr::RaggedPlan> hp(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        const fwr_plan* p = plans[i];
        hp[i].tab.tw = p->f32.tw;
        hp[i].tab.A = p->f32.A;
        hp[i].tab.Tt = p->f32.Tt;
        hp[i].tab.pt = p->f32.pt;
        hp[i].tab.iota = p->f32.iota;
        hp[i].tab.wfin = p->f32.wfin;
        hp[i].mask = p->d_mask;
        hp[i].status = p->d_status;
        hp[i].N = p->N;
        hp[i].n = p->n;
        hp[i].off = p->off;
        hp[i].periodic = p->periodic;
    }
    fwr_status st = FWR_OK;
    if ((e = cudaMalloc(&b->d_plans, sizeof(fwr::RaggedPlan) * n_plans)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_plans, hp.data(), sizeof(fwr::RaggedPlan) * n_plans, cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMalloc(&b->d_frame_plan, sizeof(int) * std::max(1, n_frames))) != cudaSuccess ||
        (n_frames > 0 && (e = cudaMemcpy(b->d_frame_plan, frame_plan, sizeof(int) * n_frames,
                                         cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMalloc(&b->d_off, sizeof(int) * (b->sms + 1))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_order, sizeof(int) * std::max(1, n_frames))) != cudaSuccess ||
        (need_scratch && (e = cudaMalloc(&b->d_scratch, size_t(b->sms) * fwr::slab_scratch_elems_per_cta(256) *
                                                            sizeof(float2))) != cudaSuccess) ||
        (e = fwr::ragged_prepare(smem)) != cudaSuccess) {
        st = fwr::cuda_fail(e, "fwr_batch_create");
    }
    cudaSetDevice(prev);
    if (st == FWR_OK) st = fwr_batch_schedule(b, b->sms, kDefaultCostRatio);
    if (st != FWR_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return FWR_OK;
}

fwr_status fwr_batch_schedule(fwr_batch* b, int ctas, double cost_ratio) {
    if (!b || ctas < 1 || ctas > b->sms || !(cost_ratio > 0.0) || !std::isfinite(cost_ratio)) return FWR_ERR_ARG;
    const int n = b->n_frames;
    std::vector<double> costs(n);
    for (int f = 0; f < n; ++f) costs[f] = b->plans[b->frame_plan[f]]->N == 256 ? cost_ratio : 1.0;
    std::vector<int> off(ctas + 1), order(std::max(1, n));
    fwr_status st = fwr_schedule_lpt(costs.data(), n, ctas, off.data(), order.data());
    if (st != FWR_OK) return st;
    // inside each CTA's list, frames of one plan run together (one table load
    // per plan and CTA)
    for (int c = 0; c < ctas; ++c)
        std::sort(order.begin() + off[c], order.begin() + off[c + 1], [&](int x, int y) {
            return b->frame_plan[x] != b->frame_plan[y] ? b->frame_plan[x] < b->frame_plan[y] : x < y;
        });
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaError_t e = cudaMemcpy(b->d_off, off.data(), sizeof(int) * (ctas + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n > 0) e = cudaMemcpy(b->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return fwr::cuda_fail(e, "fwr_batch_schedule");
    b->ctas = ctas;
    b->cost_ratio = cost_ratio;
    return FWR_OK;
}

static fwr_status batch_run(fwr_batch* b, const int* frame_plan_dev, const float* const* slopes_dev,
                            float* const* phase_dev, void* stream) {
    if (!b) return FWR_ERR_ARG;
    if (b->n_frames == 0) return FWR_OK;
    if (!slopes_dev || !phase_dev) return FWR_ERR_ARG;
    fwr::RaggedParams p;
    p.plans = b->d_plans;
    p.frame_plan = frame_plan_dev;
    p.cta_off = b->d_off;
    p.order = b->d_order;
    p.slopes = slopes_dev;
    p.phase = phase_dev;
    p.scratch = b->d_scratch;
    p.iters = b->iters;
    p.n_plans = int(b->plans.size());
    p.shape = b->shape;
    cudaError_t e = fwr::launch_ragged(p, b->ctas, b->smem, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FWR_OK : fwr::cuda_fail(e, "ragged launch");
}

fwr_status fwr_batch_run(fwr_batch* b, const float* const* slopes_dev, float* const* phase_dev, void* stream) {
    if (!b) return FWR_ERR_ARG;
    return batch_run(b, b->d_frame_plan, slopes_dev, phase_dev, stream);
}

int fwr_batch_ctas(const fwr_batch* b) { return b ? b->ctas : -1; }

int fwr_batch_shape(const fwr_batch* b) { return b ? b->shape : -1; }

fwr_status fwr_batch_set_shape(fwr_batch* b, int shape) {
    if (!b || (shape != 1 && shape != 2)) return FWR_ERR_ARG;
    b->shape = shape;
    return FWR_OK;
}

double fwr_batch_cost_ratio(const fwr_batch* b) { return b ? b->cost_ratio : -1.0; }

void fwr_batch_destroy(fwr_batch* b) {
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaFree(b->d_plans);
    cudaFree(b->d_frame_plan);
    cudaFree(b->d_off);
    cudaFree(b->d_order);
    cudaFree(b->d_scratch);
    cudaSetDevice(prev);
    delete b;
}

fwr_status fwr_batch_autotune(fwr_batch* b, const float* const* slopes_dev, float* const* phase_dev, void* stream,
                              const char* cache_path) {
    if (!b || !slopes_dev || !phase_dev) return FWR_ERR_ARG;
    // key: device, the plans' sizes and frame counts, iterations
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, b->device);
    if (e != cudaSuccess) return fwr::cuda_fail(e, "fwr_batch_autotune");
    std::vector<int> counts(b->plans.size(), 0);
    for (int f : b->frame_plan) counts[f]++;
    int drv = 0, rt = 0;
    cudaDriverGetVersion(&drv);
    cudaRuntimeGetVersion(&rt);
    bool has256 = false;
    for (const fwr_plan* pl : b->plans) has256 |= pl->N == 256;
    std::ostringstream key;
    key << prop.name << "|sm" << b->sms << "|drv" << drv << "|rt" << rt;
    for (size_t i = 0; i < b->plans.size(); ++i)
        key << "|N" << b->plans[i]->N << "n" << b->plans[i]->n << "v" << b->plans[i]->nvalid << "x" << counts[i];
    key << "|k" << b->iters;
    std::string k = key.str();
    for (char& ch : k)
        if (ch == '"' || ch == '\\') ch = '_';

    // a cached choice for this key wins (the last line for the key counts)
    if (cache_path && cache_path[0]) {
        std::ifstream in(cache_path);
        std::string line;
        int ctas = -1, shape = 2;
        double ratio = -1;
        const std::string needle = "\"key\": \"" + k + "\"";
        while (std::getline(in, line)) {
            if (line.find(needle) == std::string::npos) continue;
            size_t a = line.find("\"ctas\": "), r = line.find("\"cost_ratio\": "), sh = line.find("\"shape\": ");
            if (a == std::string::npos || r == std::string::npos) continue;
            ctas = std::atoi(line.c_str() + a + 8);
            ratio = std::atof(line.c_str() + r + 14);
            shape = sh == std::string::npos ? 2 : std::atoi(line.c_str() + sh + 9);
        }
        if (ctas >= 1 && ctas <= b->sms && ratio > 0 && (shape == 1 || shape == 2)) {
            b->shape = shape;
            return fwr_batch_schedule(b, ctas, ratio);
        }
    }

    // otherwise time the candidates on the caller's data
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return fwr::cuda_fail(e, "autotune event");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fwr::cuda_fail(e, "autotune event");
    }
    const double ratios[] = {4.0, 6.0, 8.0, 9.6, 11.0, 13.0, 16.0};
    const int ctas_opts[] = {b->sms, b->sms - b->sms / 8};
    std::vector<int> shapes = {2};
    if (has256) shapes.push_back(1);
    double best_ms = 1e30, best_ratio = kDefaultCostRatio;
    int best_ctas = b->sms, best_shape = b->shape;
    fwr_status st = FWR_OK;
    for (int shape : shapes) {
      b->shape = shape;
      for (int ctas : ctas_opts) {
        for (double ratio : ratios) {
            if ((st = fwr_batch_schedule(b, ctas, ratio)) != FWR_OK) break;
            if ((st = fwr_batch_run(b, slopes_dev, phase_dev, stream)) != FWR_OK) break;  // warm-up
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3; ++r)
                if ((st = fwr_batch_run(b, slopes_dev, phase_dev, stream)) != FWR_OK) break;
            cudaEventRecord(e1, s);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
                st = fwr::cuda_fail(e, "autotune timing");
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best_ratio = ratio;
                best_ctas = ctas;
                best_shape = shape;
            }
        }
        if (st != FWR_OK) break;
      }
      if (st != FWR_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FWR_OK) return st;
    b->shape = best_shape;
    st = fwr_batch_schedule(b, best_ctas, best_ratio);
    if (st == FWR_OK && cache_path && cache_path[0]) {
        std::ofstream o(cache_path, std::ios::app);
        o << "{\"key\": \"" << k << "\", \"ctas\": " << best_ctas << ", \"cost_ratio\": " << best_ratio
          << ", \"shape\": " << best_shape << ", \"ms_per_run\": " << best_ms / 3.0 << "}\n";
    }
    return st;
}

}  // extern "C"

// One-call ragged entry point: a schedule per (plans and their tables, frame
// table, frame count, iterations), built on first use and kept until
// fwr_ragged_release.
namespace {

struct RaggedKey {
    int device;
    std::vector<uintptr_t> plans;  // plan, its FP32 table, periodic mode, per plan
    uintptr_t frame_plan;
    int n_frames, iters;
    bool operator<(const RaggedKey& o) const {
        return std::tie(device, plans, frame_plan, n_frames, iters) <
               std::tie(o.device, o.plans, o.frame_plan, o.n_frames, o.iters);
    }
};

std::mutex g_ragged_mu;
std::map<RaggedKey, fwr_batch*> g_ragged;

}  // namespace

extern "C" {

fwr_status fwr_reconstruct_ragged(fwr_plan* const* plans, int n_plans, const int* frame_plan_dev,
                                  const float* const* slopes_dev, int n_frames, int iters, float* const* phase_dev,
                                  void* stream) {
    if (!plans || n_plans < 1 || n_frames < 0 || iters < 0 || iters > 64) return FWR_ERR_ARG;
    if (n_frames == 0) return FWR_OK;
    if (!frame_plan_dev || !slopes_dev || !phase_dev) return FWR_ERR_ARG;
    RaggedKey key;
    key.device = plans[0] ? plans[0]->device : -1;
    for (int i = 0; i < n_plans; ++i) {
        const fwr_plan* p = plans[i];
        if (!p) return FWR_ERR_ARG;
        key.plans.push_back(reinterpret_cast<uintptr_t>(p));
        key.plans.push_back(reinterpret_cast<uintptr_t>(p->f32.iota));
        key.plans.push_back(uintptr_t(p->periodic));
    }
    key.frame_plan = reinterpret_cast<uintptr_t>(frame_plan_dev);
    key.n_frames = n_frames;
    key.iters = iters;
    std::lock_guard<std::mutex> lock(g_ragged_mu);
    auto it = g_ragged.find(key);
    fwr_batch* b = nullptr;
    if (it != g_ragged.end()) {
        b = it->second;
    } else {
        // first call for this key: read the frame table (ordered after the
        // caller's earlier work on `stream`), build and keep the schedule
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        std::vector<int> fp(n_frames);
        cudaError_t e = cudaMemcpyAsync(fp.data(), frame_plan_dev, sizeof(int) * n_frames, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fwr::cuda_fail(e, "fwr_reconstruct_ragged: frame table");
        fwr_status st = fwr_batch_create(&b, plans, n_plans, fp.data(), n_frames, iters);
        if (st != FWR_OK) return st;
        g_ragged[key] = b;
    }
    return batch_run(b, frame_plan_dev, slopes_dev, phase_dev, stream);
}

void fwr_ragged_release(void) {
    std::lock_guard<std::mutex> lock(g_ragged_mu);
    for (auto& kv : g_ragged) fwr_batch_destroy(kv.second);
    g_ragged.clear();
}

}  // extern "C"
