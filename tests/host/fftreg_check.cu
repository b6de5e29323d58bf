// Host-side check of the register FFT pass arithmetic (compiled by nvcc as
// host code; no GPU): every small DFT size against the DFT definition
// X[k] = sum_n x[n] exp(-+2 pi i n k / P) in double precision, and every
// two-phase split L = P1 x P2 of the size table, run as the pass kernel runs
// it for one line (phase 1: P1-point DFTs of stride-P2 subsequences and the
// twiddles w_L^(n2 k1) from a table rounded to FP32; phase 2: P2-point DFTs;
// output k1 + P1 k2), against the length-L DFT definition.
// Exit status 0 when every relative max error is below 1e-6.
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "fftreg_impl.cuh"

using namespace ztoep;
using cd = std::complex<double>;

static double rel_err(const std::vector<cd> &ref, const std::vector<cd> &got) {
    double e = 0, n = 0;
    for (size_t i = 0; i < ref.size(); ++i) {
        e = std::max(e, std::abs(ref[i] - got[i]));
        n = std::max(n, std::abs(ref[i]));
    }
    return e / n;
}

static std::vector<cd> dft(const std::vector<cd> &x, bool inv) {
    const size_t L = x.size();
    std::vector<cd> X(L);
    for (size_t k = 0; k < L; ++k) {
        cd s = 0;
        for (size_t n = 0; n < L; ++n) {
            const double a = (inv ? 2.0 : -2.0) * M_PI * (double)((n * k) % L) / (double)L;
            s += x[n] * cd(std::cos(a), std::sin(a));
        }
        X[k] = s;
    }
    return X;
}

template <int P, bool INV> static double check_small() {
    std::mt19937 g(17 * P + INV);
    std::uniform_real_distribution<float> u(-1.f, 1.f);
    float4 v[P];
    std::vector<cd> x0(P), x1(P);
    for (int i = 0; i < P; ++i) {
        v[i] = make_float4(u(g), u(g), u(g), u(g));
        x0[i] = cd(v[i].x, v[i].y);
        x1[i] = cd(v[i].z, v[i].w);
    }
    rf::Dft<P, INV>::run(v);
    std::vector<cd> y0(P), y1(P);
    for (int i = 0; i < P; ++i) {
        y0[i] = cd(v[i].x, v[i].y);
        y1[i] = cd(v[i].z, v[i].w);
    }
    return std::max(rel_err(dft(x0, INV), y0), rel_err(dft(x1, INV), y1));
}

template <int P1, int P2, bool INV> static double check_split() {
    constexpr int L = P1 * P2;
    std::vector<float2> tw(L);
    for (int t = 0; t < L; ++t) {
        const double a = -2.0 * M_PI * t / L;
        tw[t] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    std::mt19937 g(L + INV);
    std::uniform_real_distribution<float> u(-1.f, 1.f);
    std::vector<float4> x(L), buf(L), y(L);
    for (auto &e : x) e = make_float4(u(g), u(g), u(g), u(g));
    for (int n2 = 0; n2 < P2; ++n2) {
        float4 v[P1];
        for (int n1 = 0; n1 < P1; ++n1) v[n1] = x[P2 * n1 + n2];
        rf::Dft<P1, INV>::run(v);
        for (int k1 = 1; k1 < P1; ++k1) v[k1] = rf::cmul4(v[k1], tw[n2 * k1].x, INV ? -tw[n2 * k1].y : tw[n2 * k1].y);
        for (int k1 = 0; k1 < P1; ++k1) buf[k1 * P2 + n2] = v[k1];
    }
    for (int k1 = 0; k1 < P1; ++k1) {
        float4 v[P2];
        for (int n2 = 0; n2 < P2; ++n2) v[n2] = buf[k1 * P2 + n2];
        rf::Dft<P2, INV>::run(v);
        for (int k2 = 0; k2 < P2; ++k2) y[k1 + P1 * k2] = v[k2];
    }
    std::vector<cd> x0(L), x1(L), y0(L), y1(L);
    for (int i = 0; i < L; ++i) {
        x0[i] = cd(x[i].x, x[i].y);
        x1[i] = cd(x[i].z, x[i].w);
        y0[i] = cd(y[i].x, y[i].y);
        y1[i] = cd(y[i].z, y[i].w);
    }
    return std::max(rel_err(dft(x0, INV), y0), rel_err(dft(x1, INV), y1));
}

int main() {
    double worst = 0;
    int n = 0;
#define ZT_SMALL(P)                                                         \
    {                                                                       \
        const double e = std::max(check_small<P, false>(), check_small<P, true>()); \
        std::printf("dft %d %.2e\n", P, e);                                 \
        worst = std::max(worst, e);                                         \
        ++n;                                                                \
    }
    ZT_SMALL(2) ZT_SMALL(3) ZT_SMALL(4) ZT_SMALL(5) ZT_SMALL(6) ZT_SMALL(8) ZT_SMALL(9) ZT_SMALL(10) ZT_SMALL(12)
    ZT_SMALL(15) ZT_SMALL(16)
#define ZT_SPLIT(LL, A, B)                                                                  \
    {                                                                                       \
        const double e = std::max(check_split<A, B, false>(), check_split<A, B, true>());  \
        std::printf("split %d = %d x %d %.2e\n", LL, A, B, e);                             \
        worst = std::max(worst, e);                                                         \
        ++n;                                                                                \
        if (!reg_fft_shape(LL, nullptr)) return 2;                                          \
    }
    ZT_REG_FFT_SIZES(ZT_SPLIT)
    std::printf("checked %d, worst %.2e\n", n, worst);
    return worst < 1e-6 ? 0 : 1;
}
