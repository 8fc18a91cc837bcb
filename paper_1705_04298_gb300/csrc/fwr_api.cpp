// C ABI of the reconstructor (declared in include/fwr.h): argument checks, the
// FP64 filter builder and plan-owned device tables. Every step of the
// reconstruction itself runs in the kernels of fwr_fused.cu (main path) and
// fwr_basic.cu (generic fallback for pupils too large for the main layout).

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/fwr.h"
#include "fwr_internal.h"
#include "fwr_plan.h"

namespace {

thread_local char g_last_error[256] = "";

}  // namespace

fwr_status fwr::cuda_fail(cudaError_t e, const char* where) {
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    return FWR_ERR_CUDA;
}

void fwr::set_last_error(const char* msg) { std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

namespace {
std::mutex g_setaside_mu;
std::map<int, size_t> g_setaside_before;  // device -> set-aside before the first raise
}  // namespace

void fwr::l2_setaside_note(int device, size_t before) {
    std::lock_guard<std::mutex> lock(g_setaside_mu);
    g_setaside_before.emplace(device, before);  // keeps the first value
}

bool fwr::l2_setaside_before(int device, size_t* before) {
    std::lock_guard<std::mutex> lock(g_setaside_mu);
    const auto it = g_setaside_before.find(device);
    if (it == g_setaside_before.end()) return false;
    *before = it->second;
    g_setaside_before.erase(it);
    return true;
}

namespace {
using fwr::cuda_fail;

const double kPi = 3.14159265358979323846;
const double kNullThreshold = 1e-14;

template <typename T> void free_tables(fwr::DevTables<T>& t) {
    cudaFree(t.tw);
    cudaFree(t.A);
    cudaFree(t.Tt);
    cudaFree(t.pt);
    cudaFree(t.iota);
    cudaFree(t.wfin);
    t = fwr::DevTables<T>();
}

}  // namespace

namespace {

int next_pow2(int x) {
    int p = 1;
    while (p < x) p *= 2;
    return p;
}

double signed_freq(int k, int N) { return (k < N / 2 ? double(k) : double(k - N)) / N; }

double sinc(double x) { return x == 0.0 ? 1.0 : std::sin(kPi * x) / (kPi * x); }

// FP64 filter tables (Eq. 4 model, the LSQ weight of Sec. 3.3, the Wiener
// weight of Eq. 3). Returned in the device layout of fwr::Tables.
struct HostTables {
    std::vector<double> tw, A, Tt;  // interleaved re, im; N entries each
    std::vector<double> pt;         // [N][4]: p = a conj(T) (re, im), |a|^2, |T|^2
    std::vector<double> iota, wfin; // (N/2+1) * N
};

HostTables build_tables(int N, int filter, double noise_var, double r0, double L0, int g_model, double pixel) {
    HostTables h;
    h.tw.resize(2 * N);
    h.A.resize(2 * N);
    h.Tt.resize(2 * N);
    for (int j = 0; j < N; ++j) {
        const double ang = 2.0 * kPi * double(j) / double(N);
        h.tw[2 * j] = std::cos(ang);
        h.tw[2 * j + 1] = -std::sin(ang);
        const double u = signed_freq(j, N);
        // a(u) = e^{2 i pi u} - 1; exact at u = 0 and u = -1/2. With the pixel
        // correction the difference spans d - d_px about the lenslet centre,
        // per lenslet: 2i sin(pi u L) / L e^{i pi u}, L = 1 - d_px / d (real on
        // the Nyquist bin, as G must be there)
        double ar, ai;
        if (pixel == 0.0) {
            ar = std::cos(2.0 * kPi * u) - 1.0;
            ai = std::sin(2.0 * kPi * u);
            if (j == N / 2) { ar = -2.0; ai = 0.0; }
        } else {
            const double L = 1.0 - pixel, sl = std::sin(kPi * u * L) / L;
            ar = -2.0 * sl * std::sin(kPi * u);
            ai = 2.0 * sl * std::cos(kPi * u);
            if (j == N / 2) ai = 0.0;
        }
        if (j == 0) ar = ai = 0.0;
        h.A[2 * j] = ar;
        h.A[2 * j + 1] = ai;
        // T(u) = sinc(u) e^{i pi u} (lenslet average) or cos(pi u) e^{i pi u}
        // (mean of two corner samples); the Nyquist bin takes the mean of its
        // two aliases, which is 0
        const double s = g_model == FWR_G_FRIED ? std::cos(kPi * u) : sinc(u);
        h.Tt[2 * j] = (j == N / 2) ? 0.0 : s * std::cos(kPi * u);
        h.Tt[2 * j + 1] = (j == N / 2) ? 0.0 : s * std::sin(kPi * u);
    }
    h.pt.resize(4 * size_t(N));
    for (int j = 0; j < N; ++j) {
        const double ar = h.A[2 * j], ai = h.A[2 * j + 1], tr = h.Tt[2 * j], ti = h.Tt[2 * j + 1];
        h.pt[4 * j] = ar * tr + ai * ti;      // Re a conj(T)
        h.pt[4 * j + 1] = ai * tr - ar * ti;  // Im a conj(T)
        h.pt[4 * j + 2] = ar * ar + ai * ai;
        h.pt[4 * j + 3] = tr * tr + ti * ti;
    }
    const int H = N / 2;
    h.iota.assign(size_t(H + 1) * N, 0.0);
    h.wfin.assign(size_t(H + 1) * N, 0.0);
    const double inv_n2 = 1.0 / (double(N) * double(N));  // inverse-DFT scale folded in
    const double rho = r0, ell = L0;
    for (int ky = 0; ky <= H; ++ky) {
        for (int kx = 0; kx < N; ++kx) {
            const double a2x = h.A[2 * kx] * h.A[2 * kx] + h.A[2 * kx + 1] * h.A[2 * kx + 1];
            const double a2y = h.A[2 * ky] * h.A[2 * ky] + h.A[2 * ky + 1] * h.A[2 * ky + 1];
            const double t2x = h.Tt[2 * kx] * h.Tt[2 * kx] + h.Tt[2 * kx + 1] * h.Tt[2 * kx + 1];
            const double t2y = h.Tt[2 * ky] * h.Tt[2 * ky] + h.Tt[2 * ky + 1] * h.Tt[2 * ky + 1];
            // |Gx|^2 = |a(u)|^2 |T(v)|^2, |Gy|^2 = |T(u)|^2 |a(v)|^2
            const double g2 = a2x * t2y + t2x * a2y;
            const size_t idx = size_t(ky) * N + kx;
            if (g2 < kNullThreshold) continue;
            h.iota[idx] = inv_n2 / g2;
            if (filter == FWR_WIENER) {
                const double u = signed_freq(kx, N), v = signed_freq(ky, N);
                const double kappa2 = u * u + v * v;
                const double wphi = 0.023 * std::pow(rho, -5.0 / 3.0) *
                                    std::pow(kappa2 + 1.0 / (ell * ell), -11.0 / 6.0);
                h.wfin[idx] = inv_n2 / (g2 + noise_var / wphi);
            } else {
                h.wfin[idx] = h.iota[idx];
            }
        }
    }
    return h;
}

template <typename T>
fwr_status upload_tables(const HostTables& h, int N, fwr::DevTables<T>& d) {
    typedef typename fwr::cvec<T>::type V;
    const int H = N / 2;
    std::vector<T> tw(2 * N), A(2 * N), Tt(2 * N), pt(4 * size_t(N)), iota(size_t(H + 1) * N),
        wfin(size_t(H + 1) * N);
    for (int i = 0; i < 4 * N; ++i) pt[i] = T(h.pt[i]);
    for (int i = 0; i < 2 * N; ++i) {
        tw[i] = T(h.tw[i]);
        A[i] = T(h.A[i]);
        Tt[i] = T(h.Tt[i]);
    }
    for (size_t i = 0; i < iota.size(); ++i) {
        iota[i] = T(h.iota[i]);
        wfin[i] = T(h.wfin[i]);
    }
    cudaError_t e;
    if ((e = cudaMalloc(&d.tw, N * sizeof(V))) != cudaSuccess) return cuda_fail(e, "cudaMalloc tables");
    if ((e = cudaMalloc(&d.A, N * sizeof(V))) != cudaSuccess) return cuda_fail(e, "cudaMalloc tables");
    if ((e = cudaMalloc(&d.Tt, N * sizeof(V))) != cudaSuccess) return cuda_fail(e, "cudaMalloc tables");
    if ((e = cudaMalloc(&d.pt, pt.size() * sizeof(T))) != cudaSuccess) return cuda_fail(e, "cudaMalloc tables");
    if ((e = cudaMalloc(&d.iota, iota.size() * sizeof(T))) != cudaSuccess) return cuda_fail(e, "cudaMalloc tables");
    if ((e = cudaMalloc(&d.wfin, wfin.size() * sizeof(T))) != cudaSuccess) return cuda_fail(e, "cudaMalloc tables");
    if ((e = cudaMemcpy(d.tw, tw.data(), N * sizeof(V), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d.A, A.data(), N * sizeof(V), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d.Tt, Tt.data(), N * sizeof(V), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d.pt, pt.data(), pt.size() * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d.iota, iota.data(), iota.size() * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d.wfin, wfin.data(), wfin.size() * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy tables");
    return FWR_OK;
}

template <typename T>
fwr::Tables<T> view(const fwr::DevTables<T>& d) {
    fwr::Tables<T> t;
    t.tw = d.tw;
    t.A = d.A;
    t.Tt = d.Tt;
    t.pt = d.pt;
    t.iota = d.iota;
    t.wfin = d.wfin;
    return t;
}

bool supported_grid(int N) { return N == 16 || N == 32 || N == 64 || N == 128 || N == 256 || N == 512; }


bool pow2(int N) { return N > 0 && (N & (N - 1)) == 0; }

fwr_status check_common(int n, const uint8_t* pupil_mask, int filter, double noise_var, double r0, double L0) {
    if (n < 2 || !pupil_mask) return FWR_ERR_ARG;
    if (filter != FWR_LSQ && filter != FWR_WIENER) return FWR_ERR_ARG;
    if (!(noise_var >= 0.0) || !std::isfinite(noise_var)) return FWR_ERR_ARG;
    if (filter == FWR_WIENER && (!(r0 > 0.0) || !(L0 > 0.0) || !std::isfinite(r0) || !std::isfinite(L0)))
        return FWR_ERR_ARG;
    return FWR_OK;
}

fwr_status plan_create_n(fwr_plan** out, int n, int N, const uint8_t* pupil_mask, int filter, double noise_var,
                         double r0, double L0);

}  // namespace

extern "C" {

fwr_status fwr_plan_create(fwr_plan** out, int n, double pad_factor, const uint8_t* pupil_mask, int filter,
                           double noise_var, double r0, double L0) {
    if (!out) return FWR_ERR_ARG;
    *out = nullptr;
    if (!(pad_factor >= 1.0) || !std::isfinite(pad_factor)) return FWR_ERR_ARG;
    fwr_status st = check_common(n, pupil_mask, filter, noise_var, r0, L0);
    if (st != FWR_OK) return st;
    const double want = std::ceil(pad_factor * n - 1e-9);
    if (want > 4096.0) return FWR_ERR_UNSUPPORTED;
    const int N = next_pow2(int(want));
    if (N < n + 2) return FWR_ERR_ARG;
    if (!supported_grid(N)) return FWR_ERR_UNSUPPORTED;
    return plan_create_n(out, n, N, pupil_mask, filter, noise_var, r0, L0);
}

fwr_status fwr_plan_create_grid(fwr_plan** out, int n, int N, const uint8_t* pupil_mask, int filter,
                                double noise_var, double r0, double L0) {
    if (!out) return FWR_ERR_ARG;
    *out = nullptr;
    fwr_status st = check_common(n, pupil_mask, filter, noise_var, r0, L0);
    if (st != FWR_OK) return st;
    if (N < n + 2) return FWR_ERR_ARG;
    if (pow2(N) ? !supported_grid(N) : (N % 2 != 0 || N < 16 || N > 64)) return FWR_ERR_UNSUPPORTED;
    return plan_create_n(out, n, N, pupil_mask, filter, noise_var, r0, L0);
}

}  // extern "C"

namespace {

fwr_status plan_create_n(fwr_plan** out, int n, int N, const uint8_t* pupil_mask, int filter, double noise_var,
                         double r0, double L0) {
    int nvalid = 0;
    for (int i = 0; i < n * n; ++i) nvalid += pupil_mask[i] ? 1 : 0;
    if (nvalid == 0) return FWR_ERR_ARG;

    fwr_plan* p = new (std::nothrow) fwr_plan();
    if (!p) return FWR_ERR_CUDA;
    p->n = n;
    p->N = N;
    p->off = (N - n) / 2;
    p->filter = filter;
    p->noise_var = noise_var;
    p->r0 = r0;
    p->L0 = L0;
    p->nvalid = nvalid;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaGetDevice");
    }
    std::vector<uint8_t> m(size_t(n) * n);
    for (int i = 0; i < n * n; ++i) m[i] = pupil_mask[i] ? 1 : 0;
    p->h_mask = m;
    // pupil edges of every lenslet column (first, last row) and row (first,
    // last column) for the Hudgin extension; -1 without pupil cells
    std::vector<int16_t> hud(4 * size_t(n), int16_t(-1));
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            if (!m[size_t(i) * n + j]) continue;
            if (hud[j] < 0) hud[j] = int16_t(i);
            hud[n + j] = int16_t(i);
            if (hud[2 * n + i] < 0) hud[2 * n + i] = int16_t(j);
            hud[3 * n + i] = int16_t(j);
        }
    }
    fwr_status st = FWR_OK;
    if ((e = cudaMalloc(&p->d_mask, m.size())) != cudaSuccess ||
        (e = cudaMemcpy(p->d_mask, m.data(), m.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_hud, hud.size() * sizeof(int16_t))) != cudaSuccess ||
        (e = cudaMemcpy(p->d_hud, hud.data(), hud.size() * sizeof(int16_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_status, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(p->d_status, 0, sizeof(unsigned))) != cudaSuccess) {
        st = cuda_fail(e, "plan allocation");
    }
    if (st == FWR_OK) {
        HostTables h = build_tables(N, filter, noise_var, r0, L0, p->g_model, p->pixel);
        st = upload_tables<float>(h, N, p->f32);
        if (st == FWR_OK && N <= 64) st = upload_tables<double>(h, N, p->f64);
    }
    if (st == FWR_OK && N >= 256) {
        if (fwr::slab_smem_bytes(N, n) > size_t(227) * 1024) {
            st = FWR_ERR_UNSUPPORTED;
        } else {
            p->scratch_ctas = fwr::slab_max_ctas();
            const size_t b = size_t(p->scratch_ctas) * fwr::slab_scratch_elems_per_cta(N) * sizeof(float2);
            if ((e = cudaMalloc(&p->d_scratch, b)) != cudaSuccess) st = cuda_fail(e, "cudaMalloc scratch");
            // the static array of fwr_reconstruct_static: its address on this
            // device, looked up now so that the allocation-free call itself
            // loads nothing; a failure here only disables that entry point
            if (st == FWR_OK && N == 256 && fwr::static_slab_prepare(n, &p->d_static_scratch) != cudaSuccess) {
                p->d_static_scratch = nullptr;
                cudaGetLastError();
            }
        }
    }
    if (st != FWR_OK) {
        fwr_plan_destroy(p);
        return st;
    }
    *out = p;
    return FWR_OK;
}

}  // namespace

extern "C" {

void fwr_plan_destroy(fwr_plan* p) {
    if (!p) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    free_tables(p->f32);
    free_tables(p->f64);
    cudaFree(p->d_mask);
    cudaFree(p->d_hud);
    cudaFree(p->d_status);
    cudaFree(p->d_scratch);
    cudaFree(p->d_dftws);
    cudaFree(p->d_stage_in);
    cudaFree(p->d_stage_out);
    if (p->s_h2d) cudaStreamDestroy(p->s_h2d);
    if (p->s_d2h) cudaStreamDestroy(p->s_d2h);
    for (cudaEvent_t ev : {p->ev_start, p->ev_in, p->ev_k, p->ev_done})
        if (ev) cudaEventDestroy(ev);
    cudaSetDevice(prev);
    delete p;
}

int fwr_plan_grid(const fwr_plan* p) { return p ? p->N : -1; }

int fwr_plan_valid_count(const fwr_plan* p) { return p ? p->nvalid : -1; }

// The plan's filter tables again, for its current measurement model. The new
// tables are uploaded first and replace the old ones only when complete (the
// plan keeps working tables on failure); the device is synchronised before
// the old ones are freed, since running launches may read them.
static fwr_status rebuild_tables(fwr_plan* p) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    HostTables h = build_tables(p->N, p->filter, p->noise_var, p->r0, p->L0, p->g_model, p->pixel);
    fwr::DevTables<float> t32;
    fwr::DevTables<double> t64;
    fwr_status st = upload_tables<float>(h, p->N, t32);
    if (st == FWR_OK && p->N <= 64) st = upload_tables<double>(h, p->N, t64);
    if (st == FWR_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(e, "synchronise before the table rebuild");
    }
    if (st == FWR_OK) {
        free_tables(p->f32);
        free_tables(p->f64);
        p->f32 = t32;
        p->f64 = t64;
    } else {
        free_tables(t32);
        free_tables(t64);
    }
    cudaSetDevice(prev);
    return st;
}

fwr_status fwr_plan_set_option(fwr_plan* p, int key, double value) {
    if (!p) return FWR_ERR_ARG;
    if (key == FWR_OPT_G_MODEL) {
        const int v = int(value);
        if (double(v) != value || (v != FWR_G_AVERAGED && v != FWR_G_FRIED)) return FWR_ERR_ARG;
        if (v == p->g_model) return FWR_OK;
        const int old = p->g_model;
        p->g_model = v;
        const fwr_status st = rebuild_tables(p);
        if (st != FWR_OK) p->g_model = old;
        return st;
    }
    if (key == FWR_OPT_PIXEL) {
        if (!(value >= 0.0 && value <= 0.5)) return FWR_ERR_ARG;
        if (value == p->pixel) return FWR_OK;
        const double old = p->pixel;
        p->pixel = value;
        const fwr_status st = rebuild_tables(p);
        if (st != FWR_OK) p->pixel = old;
        return st;
    }
    if (key == FWR_OPT_TRANSFORM) {
        const int v = int(value);
        if (double(v) != value ||
            (v != FWR_TRANSFORM_FFT && v != FWR_TRANSFORM_DFT_BF16X3 && v != FWR_TRANSFORM_DFT_BF16X6))
            return FWR_ERR_ARG;
        if (v == FWR_TRANSFORM_DFT_BF16X3 && p->N != 32 && p->N != 64 && p->N != 128 && p->N != 256)
            return FWR_ERR_UNSUPPORTED;  // (non-power-of-two grids included)
        if (v == FWR_TRANSFORM_DFT_BF16X6 && p->N != 64 && p->N != 128 && p->N != 256) return FWR_ERR_UNSUPPORTED;
        const int terms = v == FWR_TRANSFORM_DFT_BF16X6 ? 6 : 3;
        if (v != FWR_TRANSFORM_FFT && p->N >= 64 && (!p->d_dftws || p->dftws_terms != terms)) {
            // batched tensor-core path: its workspace is made here, not in the
            // reconstruct calls (one for the other product count is freed first,
            // after a device synchronisation)
            int prev = 0;
            cudaGetDevice(&prev);
            cudaSetDevice(p->device);
            cudaError_t e = cudaSuccess;
            if (p->d_dftws) {
                e = cudaDeviceSynchronize();
                cudaFree(p->d_dftws);
                p->d_dftws = nullptr;
                p->dftws_terms = 0;
                if (p->transform != FWR_TRANSFORM_FFT) p->transform = FWR_TRANSFORM_FFT;
            }
            if (e == cudaSuccess) e = cudaMalloc(&p->d_dftws, fwr::dftgemm_ws_bytes(p->N, terms));
            if (e == cudaSuccess) e = fwr::dftgemm_setup(p->N, terms, p->f32.tw, p->d_dftws);
            if (e != cudaSuccess) {
                cudaFree(p->d_dftws);
                p->d_dftws = nullptr;
            } else {
                p->dftws_terms = terms;
            }
            cudaSetDevice(prev);
            if (e != cudaSuccess) return cuda_fail(e, "DFT-GEMM workspace");
        }
        p->transform = v;
        return FWR_OK;
    }
    if (key == FWR_OPT_EXTENSION) {
        const int v = int(value);
        if (double(v) != value || (v != FWR_EXT_ZERO && v != FWR_EXT_HUDGIN)) return FWR_ERR_ARG;
        p->extension = v;
        return FWR_OK;
    }
    if (key == FWR_OPT_SHAPE) {
        const int v = int(value);
        if (double(v) != value || v < 0 || v > 2) return FWR_ERR_ARG;
        p->shape = v;
        return FWR_OK;
    }
    if (key == FWR_OPT_L2_PERSIST) {
        const int v = int(value);
        if (double(v) != value || (v != 0 && v != 1)) return FWR_ERR_ARG;
        if (v == 1 && !p->d_scratch) return FWR_ERR_UNSUPPORTED;
        if (v == 0) {
            p->l2_persist = 0;
            p->l2_bytes = 0;
            p->l2_hit = 0.f;
            return FWR_OK;
        }
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(p->device);
        int maxp = 0, maxw = 0;
        size_t cur = 0;
        cudaError_t e = cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, p->device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, p->device);
        if (e == cudaSuccess) e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
        const size_t scratch = size_t(p->scratch_ctas) * fwr::slab_scratch_elems_per_cta(p->N) * sizeof(float2);
        size_t want = scratch < size_t(maxp) ? scratch : size_t(maxp);
        // the context's set-aside is only raised here (other plans may use it);
        // fwr_l2_persist_reset puts back the value found before the first raise
        if (e == cudaSuccess && want > cur) {
            fwr::l2_setaside_note(p->device, cur);
            e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want);
        }
        size_t lim = 0;
        if (e == cudaSuccess) e = cudaDeviceGetLimit(&lim, cudaLimitPersistingL2CacheSize);
        cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(e, "persisting L2 set-aside");
        if (maxp <= 0 || maxw <= 0 || lim == 0) return FWR_ERR_UNSUPPORTED;
        const size_t win = scratch < size_t(maxw) ? scratch : size_t(maxw);
        p->l2_persist = 1;
        p->l2_bytes = win;
        p->l2_hit = float(double(lim) >= double(win) ? 1.0 : double(lim) / double(win));
        return FWR_OK;
    }
    if (key == FWR_OPT_CTAS) {
        const int v = int(value);
        if (double(v) != value || v < 0 || v > 65536) return FWR_ERR_ARG;
        p->ctas = v;
        return FWR_OK;
    }
    if (key == FWR_OPT_PERIODIC) {
        const int v = int(value);
        if (double(v) != value || v < FWR_PERIODIC_BEFORE_EACH_FFT || v > FWR_PERIODIC_NONE) return FWR_ERR_ARG;
        p->periodic = v;
        return FWR_OK;
    }
    return FWR_ERR_ARG;
}

static fwr_status check_call(const fwr_plan* p, const void* slopes, int n_frames, int iters, const void* phase,
                             const void* ext_out) {
    if (!p || n_frames < 0 || iters < 0 || iters > 64) return FWR_ERR_ARG;
    if (n_frames > 0 && !slopes) return FWR_ERR_ARG;
    if (n_frames > 0 && !phase && !ext_out) return FWR_ERR_ARG;
    // the phase leaves the kernels in 8- and 16-byte vector stores
    if ((reinterpret_cast<uintptr_t>(phase) & 15u) != 0) return FWR_ERR_ARG;
    return FWR_OK;
}

// the warm start is read with 16-byte vector loads (NULL passes)
static bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

fwr_status fwr_reconstruct_ex(fwr_plan* p, const float* slopes, const float* ext_init, int n_frames, int iters,
                              float* phase, float* ext_out, void* stream) {
    fwr_status st = check_call(p, slopes, n_frames, iters, phase, ext_out);
    if (st != FWR_OK) return st;
    if (!aligned16(ext_init)) return FWR_ERR_ARG;
    if (n_frames == 0) return FWR_OK;
    fwr::Params<float> k;
    k.tab = view(p->f32);
    k.mask = p->d_mask;
    k.slopes = slopes;
    k.ext_init = ext_init;
    k.phase = phase;
    k.ext_out = ext_out;
    k.n = p->n;
    k.off = p->off;
    k.F = n_frames;
    k.iters = iters;
    k.periodic = p->periodic;
    k.shape = p->shape;
    k.ctas = p->ctas;
    k.l2_bytes = p->l2_bytes;
    k.l2_hit = p->l2_hit;
    k.status = p->d_status;
    const bool hudgin = p->extension == FWR_EXT_HUDGIN && !ext_init;
    if (hudgin) {
        if (p->transform != FWR_TRANSFORM_FFT || !pow2(p->N) ||
            (p->N < 256 && !fwr::fused_supported(p->N, 4, p->n)))
            return FWR_ERR_UNSUPPORTED;
        k.hud = p->d_hud;
    }
    cudaError_t e;
    if (!pow2(p->N)) {
        e = fwr::launch_anygrid_f32(p->N, k, static_cast<cudaStream_t>(stream));
    } else if (p->transform != FWR_TRANSFORM_FFT) {
        if (p->N >= 64) {
            if (ext_out || !phase) return FWR_ERR_UNSUPPORTED;
            e = fwr::launch_dftgemm_f32(p->N, p->dftws_terms, k, p->d_dftws, static_cast<cudaStream_t>(stream));
        } else {
            e = fwr::launch_basic_gemm_f32(p->N, k, static_cast<cudaStream_t>(stream));
        }
    } else if (p->N >= 256) {
        if (ext_out || !phase) return FWR_ERR_UNSUPPORTED;
        e = fwr::launch_slab(p->N, k, p->d_scratch, p->scratch_ctas, static_cast<cudaStream_t>(stream));
    } else {
        e = fwr::fused_supported(p->N, 4, p->n) ? fwr::launch_fused_f32(p->N, k, static_cast<cudaStream_t>(stream))
                                                : fwr::launch_basic_f32(p->N, k, static_cast<cudaStream_t>(stream));
    }
    return e == cudaSuccess ? FWR_OK : cuda_fail(e, "gerchberg launch");
}

fwr_status fwr_reconstruct(fwr_plan* p, const float* slopes, int n_frames, int iters, float* phase, void* stream) {
    if (!phase && n_frames > 0) return FWR_ERR_ARG;
    return fwr_reconstruct_ex(p, slopes, nullptr, n_frames, iters, phase, nullptr, stream);
}

static_assert(FWR_STATIC_SCRATCH_GRIDS == fwr::STATIC_SLAB_GRIDS, "static scratch size mismatch");

fwr_status fwr_reconstruct_static(fwr_plan* p, const float* slopes, int n_frames, int iters, float* phase, int ctas,
                                  void* stream) {
    fwr_status st = check_call(p, slopes, n_frames, iters, phase, nullptr);
    if (st != FWR_OK) return st;
    if (!phase && n_frames > 0) return FWR_ERR_ARG;
    if (p->N != 256) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "fwr_reconstruct_static: only 256x256 grids use scratch memory (plan grid is %d)", p->N);
        return FWR_ERR_UNSUPPORTED;
    }
    if (p->transform != FWR_TRANSFORM_FFT) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "fwr_reconstruct_static: only the shared-memory FFT transform uses the static scratch "
                      "(the plan's FWR_OPT_TRANSFORM is %d)", p->transform);
        return FWR_ERR_UNSUPPORTED;
    }
    if (ctas < 1 || ctas > FWR_STATIC_SCRATCH_GRIDS) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "fwr_reconstruct_static: ctas = %d, the static scratch holds 1..%d grids of 256x256", ctas,
                      FWR_STATIC_SCRATCH_GRIDS);
        return FWR_ERR_ARG;
    }
    if (!p->d_static_scratch) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "fwr_reconstruct_static: the static scratch's device address could not be looked up when the "
                      "plan was created");
        return FWR_ERR_CUDA;
    }
    if (n_frames == 0) return FWR_OK;
    fwr::Params<float> k;
    k.tab = view(p->f32);
    k.mask = p->d_mask;
    k.slopes = slopes;
    k.ext_init = nullptr;
    k.phase = phase;
    k.ext_out = nullptr;
    k.n = p->n;
    k.off = p->off;
    k.F = n_frames;
    k.iters = iters;
    k.periodic = p->periodic;
    k.shape = p->shape;
    k.ctas = p->ctas;
    k.status = p->d_status;
    if (p->extension == FWR_EXT_HUDGIN) k.hud = p->d_hud;
    cudaError_t e = fwr::launch_slab_static(k, p->d_static_scratch, ctas, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FWR_OK : cuda_fail(e, "static-scratch launch");
}

fwr_status fwr_reconstruct_f64(fwr_plan* p, const double* slopes, const double* ext_init, int n_frames, int iters,
                               double* phase, double* ext_out, void* stream) {
    fwr_status st = check_call(p, slopes, n_frames, iters, phase, ext_out);
    if (st != FWR_OK) return st;
    if (!aligned16(ext_init)) return FWR_ERR_ARG;
    if (p->N > 64) return FWR_ERR_UNSUPPORTED;
    if (n_frames == 0) return FWR_OK;
    fwr::Params<double> k;
    k.tab = view(p->f64);
    k.mask = p->d_mask;
    k.slopes = slopes;
    k.ext_init = ext_init;
    k.phase = phase;
    k.ext_out = ext_out;
    k.n = p->n;
    k.off = p->off;
    k.F = n_frames;
    k.iters = iters;
    k.periodic = p->periodic;
    k.shape = p->shape;
    k.ctas = p->ctas;
    k.l2_bytes = p->l2_bytes;
    k.l2_hit = p->l2_hit;
    k.status = p->d_status;
    if (p->extension == FWR_EXT_HUDGIN && !ext_init) {
        if (!pow2(p->N) || !fwr::fused_supported(p->N, 8, p->n)) return FWR_ERR_UNSUPPORTED;
        k.hud = p->d_hud;
    }
    cudaError_t e = !pow2(p->N) ? fwr::launch_anygrid_f64(p->N, k, static_cast<cudaStream_t>(stream))
                    : fwr::fused_supported(p->N, 8, p->n)
                        ? fwr::launch_fused_f64(p->N, k, static_cast<cudaStream_t>(stream))
                        : fwr::launch_basic_f64(p->N, k, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FWR_OK : cuda_fail(e, "gerchberg f64 launch");
}

fwr_status fwr_plan_reserve(fwr_plan* p, int n_frames) {
    if (!p || n_frames < 0) return FWR_ERR_ARG;
    if (!p->s_h2d) {
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&p->s_h2d, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&p->s_d2h, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate (host path)");
        for (cudaEvent_t* ev : {&p->ev_start, &p->ev_in, &p->ev_k, &p->ev_done})
            if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "cudaEventCreate (host path)");
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "device attributes (host path)");
    }
    if (n_frames <= p->stage_frames) return FWR_OK;
    cudaFree(p->d_stage_in);
    cudaFree(p->d_stage_out);
    p->d_stage_in = p->d_stage_out = nullptr;
    p->stage_frames = 0;
    const size_t in_b = size_t(n_frames) * 2 * p->n * p->n * sizeof(float);
    const size_t out_b = size_t(n_frames) * p->N * p->N * sizeof(float);
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_stage_in, in_b)) != cudaSuccess) return cuda_fail(e, "cudaMalloc staging");
    if ((e = cudaMalloc(&p->d_stage_out, out_b)) != cudaSuccess) return cuda_fail(e, "cudaMalloc staging");
    p->stage_frames = n_frames;
    return FWR_OK;
}

fwr_status fwr_reconstruct_host(fwr_plan* p, const float* slopes_host, int n_frames, int iters, float* phase_host,
                                void* stream) {
    fwr_status st = check_call(p, slopes_host, n_frames, iters, phase_host, nullptr);
    if (st != FWR_OK) return st;
    if (!phase_host && n_frames > 0) return FWR_ERR_ARG;
    if (n_frames == 0) return FWR_OK;
    if ((st = fwr_plan_reserve(p, n_frames)) != FWR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t in_f = size_t(2) * p->n * p->n, out_f = size_t(p->N) * p->N;  // floats per frame
    // Pipelined in chunks of whole waves of the persistent kernel (at least two
    // SM-waves, at most four chunks): the H2D copy of chunk c + 1 and the D2H
    // copy of chunk c - 1 run on the plan's copy streams while chunk c computes
    // on `stream`; events order each chunk's copy -> kernel -> copy and join
    // the copy streams back to `stream`.
    const int wave = p->sms > 0 ? p->sms : 1;
    int chunk = (n_frames + 3) / 4;
    chunk = (chunk + wave - 1) / wave * wave;
    if (chunk < 2 * wave) chunk = 2 * wave;
    cudaError_t e;
    if ((e = cudaEventRecord(p->ev_start, s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p->s_h2d, p->ev_start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p->s_d2h, p->ev_start, 0)) != cudaSuccess)
        return cuda_fail(e, "host path ordering");
    for (int f0 = 0; f0 < n_frames; f0 += chunk) {
        const int fc = n_frames - f0 < chunk ? n_frames - f0 : chunk;
        float* din = p->d_stage_in + size_t(f0) * in_f;
        float* dout = p->d_stage_out + size_t(f0) * out_f;
        if ((e = cudaMemcpyAsync(din, slopes_host + size_t(f0) * in_f, size_t(fc) * in_f * sizeof(float),
                                 cudaMemcpyHostToDevice, p->s_h2d)) != cudaSuccess)
            return cuda_fail(e, "H2D slopes");
        if ((e = cudaEventRecord(p->ev_in, p->s_h2d)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, p->ev_in, 0)) != cudaSuccess)
            return cuda_fail(e, "host path ordering");
        st = fwr_reconstruct_ex(p, din, nullptr, fc, iters, dout, nullptr, stream);
        if (st != FWR_OK) return st;
        if ((e = cudaEventRecord(p->ev_k, s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(p->s_d2h, p->ev_k, 0)) != cudaSuccess)
            return cuda_fail(e, "host path ordering");
        if ((e = cudaMemcpyAsync(phase_host + size_t(f0) * out_f, dout, size_t(fc) * out_f * sizeof(float),
                                 cudaMemcpyDeviceToHost, p->s_d2h)) != cudaSuccess)
            return cuda_fail(e, "D2H phase");
    }
    if ((e = cudaEventRecord(p->ev_done, p->s_d2h)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, p->ev_done, 0)) != cudaSuccess)
        return cuda_fail(e, "host path ordering");
    return FWR_OK;
}

static fwr_status twiddles_for(int N, float2** out);

fwr_status fwr_dft2_bf16x3(int N, const float* in, float* out, int n_frames, int inverse, void* stream) {
    if (!(N == 32 || N == 64) || n_frames < 0) return FWR_ERR_ARG;
    if (n_frames == 0) return FWR_OK;
    if (!in || !out) return FWR_ERR_ARG;
    float2* tw = nullptr;
    fwr_status st = twiddles_for(N, &tw);
    if (st != FWR_OK) return st;
    cudaError_t e = fwr::launch_dft2_gemm_f32(N, reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out),
                                             n_frames, inverse, tw, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FWR_OK : cuda_fail(e, "dft2 bf16x3 launch");
}

fwr_status fwr_fft2(int N, const float* in, float* out, int n_frames, int inverse, void* stream) {
    if (!(N == 16 || N == 32 || N == 64 || N == 128) || n_frames < 0) return FWR_ERR_ARG;
    if (n_frames == 0) return FWR_OK;
    if (!in || !out) return FWR_ERR_ARG;
    float2* tw = nullptr;
    fwr_status st = twiddles_for(N, &tw);
    if (st != FWR_OK) return st;
    cudaError_t e = fwr::launch_fft2_f32(N, reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out),
                                        n_frames, inverse, tw, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FWR_OK : cuda_fail(e, "fft2 launch");
}

// one twiddle table per (device, N), built in FP64 and kept for the process lifetime
static fwr_status twiddles_for(int N, float2** out) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, float2*> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    float2* tw = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find({dev, N});
        if (it == cache.end()) {
            std::vector<float2> h(N);
            for (int j = 0; j < N; ++j) {
                const double ang = 2.0 * kPi * double(j) / double(N);
                h[j] = make_float2(float(std::cos(ang)), float(-std::sin(ang)));
            }
            if ((e = cudaMalloc(&tw, N * sizeof(float2))) != cudaSuccess) return cuda_fail(e, "cudaMalloc twiddles");
            if ((e = cudaMemcpy(tw, h.data(), N * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
                return cuda_fail(e, "cudaMemcpy twiddles");
            cache[{dev, N}] = tw;
        } else {
            tw = it->second;
        }
    }
    *out = tw;
    return FWR_OK;
}

fwr_status fwr_get_status(fwr_plan* p) {
    if (!p) return FWR_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    unsigned v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&v, p->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(unsigned));
    cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (v & fwr::STATUS_NONFINITE) return FWR_ERR_NONFINITE;
    if (v & fwr::STATUS_TIMEOUT) return FWR_ERR_TIMEOUT;
    if (v & fwr::STATUS_BADINDEX) return FWR_ERR_ARG;
    return FWR_OK;
}

const char* fwr_status_string(fwr_status s) {
    switch (s) {
        case FWR_OK: return "FWR_OK";
        case FWR_ERR_ARG: return "FWR_ERR_ARG";
        case FWR_ERR_UNSUPPORTED: return "FWR_ERR_UNSUPPORTED";
        case FWR_ERR_CUDA: return "FWR_ERR_CUDA";
        case FWR_ERR_NONFINITE: return "FWR_ERR_NONFINITE";
        case FWR_ERR_TIMEOUT: return "FWR_ERR_TIMEOUT";
        default: return "FWR_UNKNOWN_STATUS";
    }
}

const char* fwr_last_error(void) { return g_last_error; }

}  // extern "C"

cudaError_t fwr::launch_warm_bf16(fwr_plan* p, const float* slopes, const uint16_t* ext_init_h, int n_frames,
                                  int iters, float* phase, cudaStream_t s, bool pdl) {
    if (p->transform != FWR_TRANSFORM_FFT || p->N >= 256 || !fwr::fused_supported(p->N, 4, p->n))
        return cudaErrorNotSupported;
    fwr::Params<float> k;
    k.tab = view(p->f32);
    k.mask = p->d_mask;
    k.slopes = slopes;
    k.ext_init_h = ext_init_h;
    k.phase = phase;
    k.n = p->n;
    k.off = p->off;
    k.F = n_frames;
    k.iters = iters;
    k.periodic = p->periodic;
    k.shape = p->shape;
    k.ctas = p->ctas;
    k.status = p->d_status;
    k.pdl = pdl ? 1 : 0;
    return fwr::launch_fused_f32(p->N, k, s);
}
