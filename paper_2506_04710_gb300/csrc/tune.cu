// Autotuner: embedding sizes, FFT radix order, FFT-pass geometry, block-product
// split and tensor-core K chunk of a plan, chosen by timing the FP32 product
// on the device, with a per-process cache that can be mirrored to a file.
//
// Search (coordinate descent; the heuristic configuration is always a
// candidate, so the choice is never slower than it as measured):
//   1. embedding sizes: up to 3 x 3 (lx, ly) pairs, one plan build each;
//   2. radix order of each dimension (a plan rebuild each);
//   3. on the kept plan: FFT-pass kernel (register or shared memory) and its
//      channel batch (x threads for the shared-memory kernel) of the x passes,
//      then of the y passes, block-product split and CTAs per SM, tensor-core
//      K chunk.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "fftreg.cuh"

namespace ztoep {

void free_matvec_ws(ztoep_plan_t p);

namespace {

std::mutex g_tune_mu;
std::map<std::string, ztoep_tune_t> g_tune_cache;
bool g_file_loaded = false;

const char *cache_path() {
    const char *p = std::getenv("ZTOEP_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

// One cache line: key then the integer fields and the two times.
void load_file_locked() {
    if (g_file_loaded) return;
    g_file_loaded = true;
    const char *path = cache_path();
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (std::fgets(line, sizeof line, f)) {
        char key[512];
        ztoep_tune_t t{};
        const int n = std::sscanf(line, "%511s %d %d %d %d %d %d %d %d %d %d %d %d %d %d %lf %lf", key, &t.lx, &t.ly,
                                  &t.rad_order_x, &t.rad_order_y, &t.fft_channels_x, &t.fft_threads_x, &t.fft_channels_y,
                                  &t.fft_threads_y, &t.fft_kernel_x, &t.fft_kernel_y, &t.bp_split, &t.bp_ctas_per_sm,
                                  &t.tc_kchunk, &t.nrhs, &t.product_us, &t.default_us);
        if (n == 17) g_tune_cache[key] = t;
    }
    std::fclose(f);
}

void append_file_locked(const std::string &key, const ztoep_tune_t &t) {
    const char *path = cache_path();
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d %d %d %d %d %d %d %d %d %d %d %.3f %.3f\n", key.c_str(), t.lx, t.ly, t.rad_order_x,
                 t.rad_order_y, t.fft_channels_x, t.fft_threads_x, t.fft_channels_y, t.fft_threads_y, t.fft_kernel_x,
                 t.fft_kernel_y, t.bp_split, t.bp_ctas_per_sm, t.tc_kchunk, t.nrhs, t.product_us, t.default_us);
    std::fclose(f);
}

std::string cache_key(const ztoep_desc_t *d, int nrhs) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    std::string name(prop.name);
    for (char &c : name)
        if (c == ' ' || c == '|') c = '_';
    char buf[512];
    std::snprintf(buf, sizeof buf, "%s|sm%d|nx%d|ny%d|b%d|E%d|lx%d|ly%d|r%d", name.c_str(), prop.multiProcessorCount,
                  d->nx, d->ny, d->b, d->n_edge, d->lx, d->ly, nrhs);
    return buf;
}

int ilog2(int v) {
    int l = 0;
    while ((2 << l) <= v) ++l;
    return l;
}

TuneParams params_of(const ztoep_tune_t &t) {
    TuneParams p;
    p.rad_order[0] = t.rad_order_x;
    p.rad_order[1] = t.rad_order_y;
    p.lib[0] = t.fft_channels_x > 0 ? ilog2(t.fft_channels_x) : -1;
    p.lib[1] = t.fft_channels_y > 0 ? ilog2(t.fft_channels_y) : -1;
    p.thr[0] = t.fft_threads_x;
    p.thr[1] = t.fft_threads_y;
    p.fk[0] = t.fft_kernel_x;
    p.fk[1] = t.fft_kernel_y;
    p.bp_split = t.bp_split;
    p.bp_per_sm = t.bp_ctas_per_sm;
    p.tc_kchunk = t.tc_kchunk;
    return p;
}

void fill_tune(const ztoep_plan_t p, ztoep_tune_t *t) {
    t->lx = p->lx;
    t->ly = p->ly;
    t->rad_order_x = p->tune.rad_order[0];
    t->rad_order_y = p->tune.rad_order[1];
    t->fft_channels_x = p->tune.lib[0] >= 0 ? 1 << p->tune.lib[0] : 0;
    t->fft_channels_y = p->tune.lib[1] >= 0 ? 1 << p->tune.lib[1] : 0;
    t->fft_threads_x = p->tune.thr[0];
    t->fft_threads_y = p->tune.thr[1];
    t->fft_kernel_x = p->tune.fk[0];
    t->fft_kernel_y = p->tune.fk[1];
    t->bp_split = p->tune.bp_split;
    t->bp_ctas_per_sm = p->tune.bp_per_sm;
    t->tc_kchunk = p->tune.tc_kchunk;
}

bool pow2_or_zero(int v, int hi) { return v == 0 || (v > 0 && v <= hi && (v & (v - 1)) == 0); }

bool valid_tune(const ztoep_tune_t *t) {
    auto in = [](int v, int lo, int hi) { return v >= lo && v <= hi; };
    return in(t->rad_order_x, 0, 1) && in(t->rad_order_y, 0, 1) && pow2_or_zero(t->fft_channels_x, 64) &&
           pow2_or_zero(t->fft_channels_y, 64) && (t->fft_threads_x == 0 || t->fft_threads_x == 64 || t->fft_threads_x == 128 ||
                                       t->fft_threads_x == 256) &&
           (t->fft_threads_y == 0 || t->fft_threads_y == 64 || t->fft_threads_y == 128 || t->fft_threads_y == 256) &&
           in(t->fft_kernel_x, 0, 2) && in(t->fft_kernel_y, 0, 2) && in(t->bp_split, 0, 8) && in(t->bp_ctas_per_sm, 0, 4) && t->tc_kchunk >= 0 && t->lx >= 0 && t->ly >= 0;
}

// Mean FP32 product time (us) of `nrhs` RHS on the plan's own buffers.
ztoep_status_t time_product(ztoep_plan_t p, int nrhs, cudaStream_t s, int reps, double *us) {
    ZT_TRY(ensure_ws<float>(p, nrhs));
    ZT_TRY(ensure_tensor_data(p, nrhs, s));
    float2 *x = (float2 *)p->ws32.xin, *y = (float2 *)p->ws32.yout;
    ZT_CUDA(cudaMemsetAsync(x, 0, sizeof(float2) * (size_t)nrhs * p->N, s));
    for (int k = 0; k < 2; ++k) ZT_TRY(run_matvec<float>(p, nrhs, x, y, s));
    cudaEvent_t e0, e1;
    ZT_CUDA(cudaEventCreate(&e0));
    ZT_CUDA(cudaEventCreate(&e1));
    ztoep_status_t st = ZTOEP_OK;
    cudaEventRecord(e0, s);
    for (int k = 0; k < reps && st == ZTOEP_OK; ++k) st = run_matvec<float>(p, nrhs, x, y, s);
    cudaEventRecord(e1, s);
    const cudaError_t ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != ZTOEP_OK) return st;
    if (ce != cudaSuccess) return ZTOEP_ERR_CUDA;
    *us = 1e3 * ms / reps;
    return ZTOEP_OK;
}

// Up to three 5-smooth sizes >= 2n - 1 within 25% of the smallest (<= 256).
std::vector<int> size_candidates(int n, int fixed) {
    if (fixed) return {fixed};
    std::vector<int> c;
    const int lmin = smooth_size_at_least(2 * n - 1);
    for (int L = lmin; L <= 256 && (int)c.size() < 3 && (L <= lmin + lmin / 4 || c.empty()); ++L)
        if (is_smooth(L)) c.push_back(L);
    return c;
}

bool has_two_radices(int L) {
    const Fft1D f = make_fft1d(L, 0);
    for (int i = 1; i < f.nst; ++i)
        if (f.rad[i] != f.rad[0]) return true;
    return false;
}

int reps_for(double us) { return us < 200 ? 20 : (us < 2000 ? 8 : 3); }

}  // namespace
}  // namespace ztoep

using namespace ztoep;

extern "C" {

ztoep_status_t ztoep_plan_get_tune(ztoep_plan_t p, ztoep_tune_t *t) {
    if (!p || !t) return ZTOEP_ERR_ARG;
    std::memset(t, 0, sizeof *t);
    fill_tune(p, t);
    return ZTOEP_OK;
}

ztoep_status_t ztoep_plan_tuned(const ztoep_desc_t *desc, const void *T, const void *B, const void *C,
                                const ztoep_tune_t *tune, void *stream, ztoep_plan_t *out) {
    if (!desc || !tune || !out || !valid_tune(tune)) return ZTOEP_ERR_ARG;
    ztoep_desc_t d = *desc;
    if (tune->lx) d.lx = tune->lx;
    if (tune->ly) d.ly = tune->ly;
    return plan_create(&d, T, B, C, (cudaStream_t)stream, params_of(*tune), out);
}

ztoep_status_t ztoep_plan_autotune(const ztoep_desc_t *desc, const void *T, const void *B, const void *C,
                                   int32_t nrhs, void *stream, ztoep_plan_t *out, ztoep_tune_t *tune) {
    if (!desc || !out || nrhs < 1 || nrhs > kTcMaxRhs) return ZTOEP_ERR_ARG;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key = cache_key(desc, nrhs);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_file_locked();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            ztoep_tune_t t = it->second;
            t.candidates = 0;
            ZT_TRY(ztoep_plan_tuned(desc, T, B, C, &t, stream, out));
            if (tune) *tune = t;
            return ZTOEP_OK;
        }
    }
    int timed = 0;
    double best_us = 0, default_us = 0;
    ztoep_plan_t best = nullptr;
    auto consider = [&](ztoep_plan_t q, double us) {  // keeps the faster of best and q
        if (!best || us < best_us) {
            if (best) ztoep_plan_destroy(best);
            best = q;
            best_us = us;
        } else {
            ztoep_plan_destroy(q);
        }
    };
    auto fail = [&](ztoep_status_t st) {
        if (best) ztoep_plan_destroy(best);
        return st;
    };
    // 1. embedding sizes
    const std::vector<int> cx = size_candidates(desc->nx, desc->lx), cy = size_candidates(desc->ny, desc->ly);
    for (int lx : cx)
        for (int ly : cy) {
            ztoep_desc_t d = *desc;
            d.lx = lx;
            d.ly = ly;
            ztoep_plan_t q = nullptr;
            ztoep_status_t st = plan_create(&d, T, B, C, s, TuneParams{}, &q);
            if (st != ZTOEP_OK) return fail(st);
            double us = 0;
            st = time_product(q, nrhs, s, 10, &us);
            if (st != ZTOEP_OK) {
                ztoep_plan_destroy(q);
                return fail(st);
            }
            ++timed;
            if (lx == cx[0] && ly == cy[0]) default_us = us;
            consider(q, us);
        }
    const int reps = reps_for(best_us);
    // 2. radix order per dimension (rebuilds)
    for (int dim = 0; dim < 2; ++dim) {
        if (!has_two_radices(dim == 0 ? best->lx : best->ly)) continue;
        TuneParams tp = best->tune;
        tp.rad_order[dim] = 1;
        ztoep_desc_t d = *desc;
        d.lx = best->lx;
        d.ly = best->ly;
        ztoep_plan_t q = nullptr;
        ztoep_status_t st = plan_create(&d, T, B, C, s, tp, &q);
        if (st != ZTOEP_OK) return fail(st);
        double us = 0;
        st = time_product(q, nrhs, s, reps, &us);
        if (st != ZTOEP_OK) {
            ztoep_plan_destroy(q);
            return fail(st);
        }
        ++timed;
        consider(q, us);
    }
    // 3. launch shapes on the kept plan
    auto try_params = [&](const TuneParams &tp, bool realloc) -> ztoep_status_t {
        const TuneParams keep = best->tune;
        best->tune = tp;
        if (realloc) free_matvec_ws(best);
        double us = 0;
        ZT_TRY(time_product(best, nrhs, s, reps, &us));
        ++timed;
        if (us < best_us) {
            best_us = us;
        } else {
            best->tune = keep;
            if (realloc) free_matvec_ws(best);
        }
        return ZTOEP_OK;
    };
    for (int dim = 0; dim < 2; ++dim) {
        const int L = dim == 0 ? best->lx : best->ly;
        const int lines = dim == 0 ? best->ny * nrhs : best->lx * nrhs;
        const bool reg = reg_fft_shape(L, nullptr);
        if (reg) {  // register kernel (the heuristic): channel batches 8..64
            const int h = 2 * reg_fft_cpb(L, best->b, lines, best->nsm, 0);
            for (int ch = 8; ch <= 64; ch *= 2) {
                if (ch == h || 2 * reg_fft_cpb(L, best->b, lines, best->nsm, ch) != ch) continue;
                TuneParams tp = best->tune;
                tp.fk[dim] = 2;
                tp.lib[dim] = ilog2(ch);
                ztoep_status_t st = try_params(tp, false);
                if (st != ZTOEP_OK) return fail(st);
            }
        }
        // shared-memory kernel: its heuristic, then channel batch x threads around it
        const PassCfg h = pass_cfg(L, best->b, lines, sizeof(float2), best->nsm);
        const int maxlib = pick_lib(L, best->b, sizeof(float2), 64 * 1024);
        for (int lib = std::max(0, h.lib - 1); lib <= std::min(maxlib, h.lib + 1); ++lib)
            for (int thr : {64, 128, 256}) {
                if (!reg && lib == h.lib && thr == h.threads) continue;  // the heuristic itself
                TuneParams tp = best->tune;
                tp.fk[dim] = 1;
                tp.lib[dim] = lib;
                tp.thr[dim] = thr;
                ztoep_status_t st = try_params(tp, false);
                if (st != ZTOEP_OK) return fail(st);
            }
    }
    if (nrhs < kTcMinRhs) {
        for (int S : {1, 2, 4, 8}) {
            if (best->b % S) continue;
            TuneParams tp = best->tune;
            tp.bp_split = S;
            ztoep_status_t st = try_params(tp, false);
            if (st != ZTOEP_OK) return fail(st);
        }
        for (int per_sm = 1; per_sm <= 4; ++per_sm) {
            TuneParams tp = best->tune;
            tp.bp_per_sm = per_sm;
            ztoep_status_t st = try_params(tp, false);
            if (st != ZTOEP_OK) return fail(st);
        }
    } else if (best->E > 0 && best->side_k == 0) {
        const int mt = (best->E + 63) / 64;
        const int want = std::max(1, (2 * best->nsm + mt - 1) / mt);
        const int kc0 = std::max(256, (int)((best->NT + want - 1) / want + 15) / 16 * 16);
        for (int kc : {kc0 / 2, kc0 * 2, kc0 * 4}) {
            if (kc < 64) continue;
            TuneParams tp = best->tune;
            tp.tc_kchunk = kc;
            ztoep_status_t st = try_params(tp, true);
            if (st != ZTOEP_OK) return fail(st);
        }
    }
    free_solve_graphs(best);
    ztoep_tune_t t{};
    fill_tune(best, &t);
    t.nrhs = nrhs;
    t.candidates = timed;
    t.product_us = best_us;
    t.default_us = default_us;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = t;
        append_file_locked(key, t);
    }
    if (tune) *tune = t;
    *out = best;
    return ZTOEP_OK;
}

}  // extern "C"
