// Launch-shape tuning of a plan (fwr_plan_autotune, include/fwr.h): times the
// kernel shapes and persistent-grid sizes a plan's grid offers on the
// caller's data and keeps the fastest, with a JSON-lines cache keyed by the
// device, the driver and runtime versions and the problem. The candidates
// differ only in how the work is laid out on the GPU; every one gives
// bitwise the same result.

#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/fwr.h"
#include "fwr_internal.h"
#include "fwr_plan.h"

namespace {

std::string tune_key(const fwr_plan* p, int n_frames, int iters) {
    cudaDeviceProp prop;
    int drv = 0, rt = 0, sms = 0;
    if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) prop.name[0] = 0;
    cudaDriverGetVersion(&drv);
    cudaRuntimeGetVersion(&rt);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    std::ostringstream k;
    k << prop.name << "|sm" << sms << "|drv" << drv << "|rt" << rt << "|N" << p->N << "n" << p->n << "v"
      << p->nvalid << "|t" << p->transform << "p" << p->periodic << "f" << p->filter << "e" << p->extension << "g"
      << p->g_model << "x" << p->pixel << "|F" << n_frames << "|k" << iters;
    std::string s = k.str();
    for (char& ch : s)
        if (ch == '"' || ch == '\\') ch = '_';
    return s;
}

// the last cached (shape, ctas, l2_persist) for a key; false if none
bool cached(const char* path, const std::string& key, int* shape, int* ctas, int* persist) {
    if (!path || !path[0]) return false;
    std::ifstream in(path);
    std::string line;
    const std::string needle = "\"key\": \"" + key + "\"";
    bool found = false;
    while (std::getline(in, line)) {
        if (line.find(needle) == std::string::npos) continue;
        const size_t a = line.find("\"shape\": "), c = line.find("\"ctas\": ");
        if (a == std::string::npos || c == std::string::npos) continue;
        *shape = std::atoi(line.c_str() + a + 9);
        *ctas = std::atoi(line.c_str() + c + 8);
        const size_t l = line.find("\"l2_persist\": ");
        *persist = l == std::string::npos ? 0 : std::atoi(line.c_str() + l + 14);
        found = true;
    }
    return found && *shape >= 0 && *shape <= 2 && *ctas >= 0;
}

}  // namespace

extern "C" {

int fwr_plan_shape(const fwr_plan* p) { return p ? p->shape : -1; }

int fwr_plan_ctas(const fwr_plan* p) { return p ? p->ctas : -1; }

int fwr_plan_l2_persist(const fwr_plan* p) { return p ? p->l2_persist : -1; }

fwr_status fwr_l2_persist_reset(int device) {
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return FWR_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaError_t e = cudaCtxResetPersistingL2Cache();
    size_t before = 0;
    if (e == cudaSuccess && fwr::l2_setaside_before(device, &before))
        e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, before);
    cudaSetDevice(prev);
    return e == cudaSuccess ? FWR_OK : fwr::cuda_fail(e, "fwr_l2_persist_reset");
}

fwr_status fwr_plan_autotune(fwr_plan* p, const float* slopes, int n_frames, int iters, float* phase, void* stream,
                             const char* cache_path) {
    if (!p || !slopes || !phase || n_frames < 1 || iters < 0 || iters > 64) return FWR_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    const std::string key = tune_key(p, n_frames, iters);
    int shape = 0, ctas = 0, persist = 0;
    if (cached(cache_path, key, &shape, &ctas, &persist)) {
        p->shape = shape;
        p->ctas = ctas;
        fwr_status st = FWR_OK;
        if (persist != p->l2_persist) st = fwr_plan_set_option(p, FWR_OPT_L2_PERSIST, persist);
        cudaSetDevice(prev);
        return st == FWR_ERR_UNSUPPORTED ? FWR_OK : st;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    // shapes: two for 256^2 (warp groups) and for the fused FFT kernels
    // (final weights in shared memory or L2); the DFT-GEMM transform and the
    // other kernels have one
    std::vector<int> shapes = {0};
    const bool fft = p->transform == FWR_TRANSFORM_FFT;
    if (fft && p->N == 256) shapes = {2, 1};
    else if (fft && (p->N & (p->N - 1)) == 0 && p->N <= 128) shapes = {1, 2};
    // the plan's L2 window (FWR_OPT_L2_PERSIST) stays as the caller set it:
    // its set-aside changes the L2 for everything else the process runs, which
    // timing the plan alone cannot weigh
    std::vector<int> persist_opts = {p->l2_persist};
    std::vector<int> ctas_opts = {0};
    if (sms >= 8) {
        ctas_opts.push_back(3 * sms / 4);
        ctas_opts.push_back(sms / 2);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaSetDevice(prev);
        return fwr::cuda_fail(e, "fwr_plan_autotune events");
    }
    const int old_shape = p->shape, old_ctas = p->ctas, old_persist = p->l2_persist;
    double best = 1e30;
    int best_shape = old_shape, best_ctas = old_ctas, best_persist = old_persist;
    fwr_status st = FWR_OK;
    for (int pe : persist_opts) {
      if (pe != p->l2_persist && (st = fwr_plan_set_option(p, FWR_OPT_L2_PERSIST, pe)) != FWR_OK) {
          if (st == FWR_ERR_UNSUPPORTED) {  // no persisting L2 on this device: skip the candidate
              st = FWR_OK;
              continue;
          }
          break;
      }
      for (int sh : shapes) {
        for (int c : ctas_opts) {
            p->shape = sh;
            p->ctas = c;
            if ((st = fwr_reconstruct_ex(p, slopes, nullptr, n_frames, iters, phase, nullptr, stream)) != FWR_OK)
                break;  // warm-up
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3 && st == FWR_OK; ++r)
                st = fwr_reconstruct_ex(p, slopes, nullptr, n_frames, iters, phase, nullptr, stream);
            cudaEventRecord(e1, s);
            if (st != FWR_OK) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
                st = fwr::cuda_fail(e, "fwr_plan_autotune timing");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_shape = sh;
                best_ctas = c;
                best_persist = pe;
            }
        }
        if (st != FWR_OK) break;
      }
      if (st != FWR_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FWR_OK) {
        p->shape = old_shape;
        p->ctas = old_ctas;
        fwr_plan_set_option(p, FWR_OPT_L2_PERSIST, old_persist);
        cudaSetDevice(prev);
        return st;
    }
    p->shape = best_shape;
    p->ctas = best_ctas;
    if (best_persist != p->l2_persist) fwr_plan_set_option(p, FWR_OPT_L2_PERSIST, best_persist);
    if (cache_path && cache_path[0]) {
        std::ofstream o(cache_path, std::ios::app);
        o << "{\"key\": \"" << key << "\", \"shape\": " << best_shape << ", \"ctas\": " << best_ctas
          << ", \"l2_persist\": " << best_persist << ", \"ms_per_run\": " << best / 3.0 << "}\n";
    }
    cudaSetDevice(prev);
    return FWR_OK;
}

}  // extern "C"
