// CPU FFT baseline: the Gerchberg extension loop and Fourier reconstructor
// (Algorithm 1 of Sec. 3.3 with the periodic condition Eq. PC, the LSQ
// projection inside the loop and the Wiener or LSQ final filter of Eqs. 2-3)
// with a radix-2 FFT, in FP64 or FP32, one frame per host thread.
//
// This is a timing baseline, not part of the library: bench.py reports it
// beside the direct-DFT oracle (a fairer CPU comparison than an O(N^3) DFT),
// and the tests check it against the oracle. It shares no code with the
// CUDA library or with the oracle.
//
// Per frame: the x and y slopes are packed into one complex grid
// Z = sx + i sy; each iteration takes one forward and one inverse 2-D FFT.
// The spectral step unpacks the bin pair (k, -k):
//   Sx = (Z(k) + conj Z(-k)) / 2,  Sy = (Z(k) - conj Z(-k)) / (2i),
// forms the LSQ phase phi = (conj Gx Sx + conj Gy Sy) / |G|^2 and
// re-synthesises Z'(k) = Gx phi + i Gy phi. The measurement model is the
// lenslet-averaged gradient Gx = a(u) T(v), Gy = T(u) a(v) with
// a(u) = e^{2 i pi u} - 1 and T(u) = sinc(u) e^{i pi u}, T = 0 on the Nyquist
// bin, 1/|G|^2 = 0 where |G|^2 < 1e-14 (piston and waffle).

#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;

template <typename T> struct Fft {
    int N = 0, logN = 0;
    std::vector<std::complex<T>> w;  // e^{-2 i pi j / N}, j < N/2
    std::vector<int> rev;

    explicit Fft(int n) : N(n) {
        while ((1 << logN) < N) ++logN;
        w.resize(N / 2);
        for (int j = 0; j < N / 2; ++j) {
            const double a = 2.0 * kPi * double(j) / double(N);
            w[j] = std::complex<T>(T(std::cos(a)), T(-std::sin(a)));
        }
        rev.resize(N);
        for (int i = 0; i < N; ++i) {
            int r = 0;
            for (int b = 0; b < logN; ++b) r |= ((i >> b) & 1) << (logN - 1 - b);
            rev[i] = r;
        }
    }

    // in-place radix-2 decimation-in-time transform of one line; inverse uses
    // the conjugate twiddles and no scaling
    void line(std::complex<T>* x, bool inverse) const {
        for (int i = 0; i < N; ++i)
            if (i < rev[i]) std::swap(x[i], x[rev[i]]);
        for (int h = 1; h < N; h *= 2) {
            const int step = N / (2 * h);
            for (int b = 0; b < N; b += 2 * h) {
                for (int j = 0; j < h; ++j) {
                    std::complex<T> t = w[j * step];
                    if (inverse) t = std::conj(t);
                    const std::complex<T> u = x[b + j], v = t * x[b + j + h];
                    x[b + j] = u + v;
                    x[b + j + h] = u - v;
                }
            }
        }
    }

    // 2-D transform of an N x N grid (rows, transpose, rows, transpose)
    void grid(std::complex<T>* z, std::complex<T>* tmp, bool inverse) const {
        for (int r = 0; r < N; ++r) line(z + size_t(r) * N, inverse);
        for (int r = 0; r < N; ++r)
            for (int c = 0; c < N; ++c) tmp[size_t(c) * N + r] = z[size_t(r) * N + c];
        for (int r = 0; r < N; ++r) line(tmp + size_t(r) * N, inverse);
        for (int r = 0; r < N; ++r)
            for (int c = 0; c < N; ++c) z[size_t(c) * N + r] = tmp[size_t(r) * N + c];
    }
};

struct Model {
    int N = 0;
    std::vector<std::complex<double>> a, t;  // a(u), T(u) per frequency index
    std::vector<double> iota, wfin;          // 1/|G|^2 and the final weight per bin (N x N)
};

Model build_model(int N, int filter, double noise_var, double r0, double L0) {
    Model m;
    m.N = N;
    m.a.resize(N);
    m.t.resize(N);
    for (int j = 0; j < N; ++j) {
        const double u = (j < N / 2 ? double(j) : double(j - N)) / double(N);
        m.a[j] = std::complex<double>(std::cos(2 * kPi * u) - 1.0, std::sin(2 * kPi * u));
        if (j == N / 2) m.a[j] = std::complex<double>(-2.0, 0.0);
        if (j == 0) m.a[j] = 0.0;
        const double s = u == 0.0 ? 1.0 : std::sin(kPi * u) / (kPi * u);
        m.t[j] = (j == N / 2) ? std::complex<double>(0.0, 0.0)
                              : std::complex<double>(s * std::cos(kPi * u), s * std::sin(kPi * u));
    }
    m.iota.assign(size_t(N) * N, 0.0);
    m.wfin.assign(size_t(N) * N, 0.0);
    for (int ky = 0; ky < N; ++ky) {
        for (int kx = 0; kx < N; ++kx) {
            const double g2 = std::norm(m.a[kx] * m.t[ky]) + std::norm(m.t[kx] * m.a[ky]);
            if (g2 < 1e-14) continue;
            const size_t i = size_t(ky) * N + kx;
            m.iota[i] = 1.0 / g2;
            if (filter == 1) {
                const double u = (kx < N / 2 ? double(kx) : double(kx - N)) / double(N);
                const double v = (ky < N / 2 ? double(ky) : double(ky - N)) / double(N);
                const double wphi = 0.023 * std::pow(r0, -5.0 / 3.0) * std::pow(u * u + v * v + 1.0 / (L0 * L0),
                                                                                 -11.0 / 6.0);
                m.wfin[i] = 1.0 / (g2 + noise_var / wphi);
            } else {
                m.wfin[i] = m.iota[i];
            }
        }
    }
    return m;
}

// Eq. PC on the packed grid: last column of x = -(sum of the row's others),
// last row of y = -(sum of the column's others)
template <typename T> void periodic_fill(std::complex<T>* z, int N) {
    for (int r = 0; r < N; ++r) {
        T s = 0;
        for (int c = 0; c < N - 1; ++c) s += z[size_t(r) * N + c].real();
        z[size_t(r) * N + N - 1].real(-s);
    }
    for (int c = 0; c < N; ++c) {
        T s = 0;
        for (int r = 0; r < N - 1; ++r) s += z[size_t(r) * N + c].imag();
        z[size_t(N - 1) * N + c].imag(-s);
    }
}

template <typename T> struct Frame {
    const Model& m;
    const Fft<T>& fft;
    std::vector<std::complex<T>> z, tmp, out;
    std::vector<std::complex<T>> gx, gy;  // Gx, Gy per bin in T
    std::vector<T> iota, wfin;
    Frame(const Model& mm, const Fft<T>& f) : m(mm), fft(f) {
        const int N = m.N;
        z.resize(size_t(N) * N);
        tmp.resize(size_t(N) * N);
        out.resize(size_t(N) * N);
        gx.resize(size_t(N) * N);
        gy.resize(size_t(N) * N);
        iota.resize(size_t(N) * N);
        wfin.resize(size_t(N) * N);
        for (int ky = 0; ky < N; ++ky)
            for (int kx = 0; kx < N; ++kx) {
                const size_t i = size_t(ky) * N + kx;
                const std::complex<double> a = m.a[kx] * m.t[ky], b = m.t[kx] * m.a[ky];
                gx[i] = std::complex<T>(T(a.real()), T(a.imag()));
                gy[i] = std::complex<T>(T(b.real()), T(b.imag()));
                iota[i] = T(m.iota[i]);
                wfin[i] = T(m.wfin[i]);
            }
    }

    // spectral step on the packed spectrum z (into out): LSQ projection when
    // final is false, the final filter's phase spectrum otherwise
    void spectral(bool final) {
        const int N = m.N;
        const T half = T(0.5);
        for (int ky = 0; ky < N; ++ky) {
            const int ny = (N - ky) & (N - 1);
            for (int kx = 0; kx < N; ++kx) {
                const int nx = (N - kx) & (N - 1);
                const size_t i = size_t(ky) * N + kx;
                const std::complex<T> z1 = z[i], z2 = std::conj(z[size_t(ny) * N + nx]);
                const std::complex<T> sx = (z1 + z2) * half;
                const std::complex<T> sy = (z1 - z2) * std::complex<T>(0, -half);
                const std::complex<T> ph = std::conj(gx[i]) * sx + std::conj(gy[i]) * sy;
                if (final) {
                    out[i] = ph * wfin[i];
                } else {
                    const std::complex<T> p = ph * iota[i];
                    out[i] = gx[i] * p + std::complex<T>(0, 1) * (gy[i] * p);
                }
            }
        }
    }

    void run(const double* sl, const uint8_t* mask, int n, int iters, int periodic, double* phase) {
        const int N = m.N, off = (N - n) / 2;
        const T scale = T(1.0 / (double(N) * double(N)));
        std::fill(z.begin(), z.end(), std::complex<T>(0, 0));
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (mask[i * n + j])
                    z[size_t(off + i) * N + off + j] = std::complex<T>(T(sl[i * n + j]), T(sl[n * n + i * n + j]));
        for (int it = 0; it <= iters; ++it) {
            const bool final = it == iters;
            if (periodic == 0 || (periodic == 1 && final)) periodic_fill(z.data(), N);
            fft.grid(z.data(), tmp.data(), false);
            spectral(final);
            fft.grid(out.data(), tmp.data(), true);
            if (!final) {
                for (size_t c = 0; c < z.size(); ++c) z[c] = out[c] * scale;
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j)
                        if (mask[i * n + j])
                            z[size_t(off + i) * N + off + j] =
                                std::complex<T>(T(sl[i * n + j]), T(sl[n * n + i * n + j]));
            } else {
                for (size_t c = 0; c < z.size(); ++c) phase[c] = double(out[c].real() * scale);
            }
        }
    }
};

template <typename T>
void run_all(const Model& m, const double* slopes, int F, int n, const uint8_t* mask, int iters, int periodic,
             double* phase, int threads) {
    const Fft<T> fft(m.N);
    std::atomic<int> next(0);
    auto worker = [&]() {
        Frame<T> fr(m, fft);
        for (int f = next++; f < F; f = next++)
            fr.run(slopes + size_t(f) * 2 * n * n, mask, n, iters, periodic, phase + size_t(f) * m.N * m.N);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
}

}  // namespace

extern "C" {

// slopes [F][2][n][n] (x then y), mask [n][n] (nonzero = valid), phase
// [F][N][N] out (zero mean); N a power of two >= n + 2; precision 32 or 64;
// filter 0 = LSQ, 1 = Wiener (noise_var rad^2, r0 and L0 in lenslet
// pitches); periodic 0 = before every forward FFT, 1 = before the final one
// only, 2 = never; threads <= 0: all hardware threads. Returns 0, or -1 for a
// bad argument.
int fwr_cpu_fft_reconstruct(int precision, const double* slopes, int F, int n, const uint8_t* mask, int N,
                            int iters, int filter, double noise_var, double r0, double L0, int periodic,
                            double* phase, int threads) {
    if (F < 0 || n < 2 || N < n + 2 || (N & (N - 1)) != 0 || iters < 0 || periodic < 0 || periodic > 2 ||
        (precision != 32 && precision != 64) || !slopes || !mask || !phase)
        return -1;
    if (threads <= 0) threads = int(std::thread::hardware_concurrency());
    if (threads < 1) threads = 1;
    if (threads > F) threads = F > 0 ? F : 1;
    const Model m = build_model(N, filter, noise_var, r0, L0);
    if (precision == 64) run_all<double>(m, slopes, F, n, mask, iters, periodic, phase, threads);
    else run_all<float>(m, slopes, F, n, mask, iters, periodic, phase, threads);
    return 0;
}

int fwr_cpu_fft_threads(void) { return int(std::thread::hardware_concurrency()); }

}  // extern "C"
