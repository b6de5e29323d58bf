// Plan construction: circulant embedding of the generating blocks of the
// two-level block-Toeplitz matrix A (Eq. submatrixAA), their 2-D FFT over the
// element indices (FP64), resident storage of one transformed block per
// frequency pair {f, -f} (Z = Z^T, Sec. II-A, gives T^(-f) = T^(f)^T), and the
// edge-coupling blocks B and C (Eq. matrixForm).  Also the C-ABI entry points
// for the matvec and the inspection calls.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "instrument.cuh"

namespace ztoep {

void free_matvec_ws(ztoep_plan_t p);
void free_solve_ws(ztoep_plan_t p);
int64_t edge_row_stride(int64_t NT);
int64_t edge_row_stride32(int64_t NT, int E);
ztoep_status_t pack_bc32(ztoep_plan_t p, cudaStream_t s);

bool is_smooth(int n) {
    if (n < 1) return false;
    for (int q : {2, 3, 5})
        while (n % q == 0) n /= q;
    return n == 1;
}

int smooth_size_at_least(int n) {
    int L = std::max(1, n);
    while (!is_smooth(L)) ++L;
    return L;
}

Fft1D make_fft1d(int L, int order) {
    Fft1D f{};
    f.L = L;
    int n = L;
    while (n % 4 == 0) { f.rad[f.nst++] = 4; n /= 4; }
    while (n % 2 == 0) { f.rad[f.nst++] = 2; n /= 2; }
    while (n % 3 == 0) { f.rad[f.nst++] = 3; n /= 3; }
    while (n % 5 == 0) { f.rad[f.nst++] = 5; n /= 5; }
    if (order == 1)
        for (int i = 0, j = f.nst - 1; i < j; ++i, --j) std::swap(f.rad[i], f.rad[j]);
    int Ns = 1;
    for (int s = 0; s < f.nst; ++s) {
        f.ns[s] = Ns;
        f.mag[s] = 65536 / Ns + 1;
        Ns *= f.rad[s];
    }
    return f;
}

ztoep_status_t dalloc(void **p, size_t bytes, size_t *acc) {
    *p = nullptr;
    if (bytes == 0) return ZTOEP_OK;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return ZTOEP_ERR_NOMEM;
    }
    if (acc) *acc += bytes;
    return ZTOEP_OK;
}

// ------------------------------------------------------------ plan FFT functors
// Channels c = (i, j) of the b x b blocks, c < b*b.
struct LdPlanX {  // row qi of T (offset q = qi - ny + 1); position kx <- offset p, p mod lx
    const double2 *T; int nx, lx, bb, ib;
    __device__ double2 operator()(int pos, int ch) const {
        const int qi = blockIdx.y, c = blockIdx.x * ib + ch;
        if (c >= bb) return czero<double2>();
        const int p = pos < nx ? pos : pos - lx;
        if (p <= -nx || p >= nx) return czero<double2>();
        return T[((int64_t)qi * (2 * nx - 1) + (p + nx - 1)) * bb + c];
    }
};
struct StPlanX {
    double2 *P1; int lx, bb, ib;
    __device__ void operator()(int kx, int ch, double2 v) const {
        const int qi = blockIdx.y, c = blockIdx.x * ib + ch;
        if (c < bb) P1[((int64_t)qi * lx + kx) * bb + c] = v;
    }
};
struct LdPlanY {  // column kx; position ky <- offset q, q mod ly
    const double2 *P1; int ny, ly, lx, bb, ib;
    __device__ double2 operator()(int pos, int ch) const {
        const int kx = blockIdx.y, c = blockIdx.x * ib + ch;
        if (c >= bb) return czero<double2>();
        const int q = pos < ny ? pos : pos - ly;
        if (q <= -ny || q >= ny) return czero<double2>();
        return P1[((int64_t)(q + ny - 1) * lx + kx) * bb + c];
    }
};
struct StPlanY {  // keep the stored representative of each pair, FP64 and FP32
    const int *rep; double2 *T64; float2 *T32; int lx, bb, ib;
    __device__ void operator()(int ky, int ch, double2 v) const {
        const int kx = blockIdx.y, c = blockIdx.x * ib + ch;
        if (c >= bb) return;
        const int pi = rep[ky * lx + kx];
        if (pi < 0) return;
        T64[(int64_t)pi * bb + c] = v;
        T32[(int64_t)pi * bb + c] = make_float2((float)v.x, (float)v.y);
    }
};

__global__ void k_zero_columns(double2 *B, int64_t ldb, int E, const uint8_t *active, int nel, int b) {
    // B[e][el*b + i] = 0 for absent elements el
    const int64_t total = (int64_t)E * nel * b;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = k / ((int64_t)nel * b);
        const int64_t t = k - e * nel * b;
        if (!active[t / b]) B[e * ldb + t] = czero<double2>();
    }
}

__global__ void k_expand_spectrum(const double2 *__restrict__ T64, const int *__restrict__ rep, double2 *out,
                                  int F, int b) {
    const int64_t bb = (int64_t)b * b;
    const int64_t total = (int64_t)F * bb;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(k / bb);
        const int64_t c = k - f * bb;
        const int i = (int)(c / b), j = (int)(c - (int64_t)i * b);
        const int r = rep[f];
        out[k] = r >= 0 ? T64[(int64_t)r * bb + c] : T64[(int64_t)(-1 - r) * bb + (int64_t)j * b + i];
    }
}

static bool valid_desc(const ztoep_desc_t *d) {
    if (!d) return false;
    if (d->nx < 1 || d->ny < 1 || d->b < 1 || d->b > 128 || d->n_edge < 0) return false;
    if (d->nx > 4096 || d->ny > 4096) return false;
    if (d->lx != 0 && (d->lx < 2 * d->nx - 1 || d->lx > 256 || !is_smooth(d->lx))) return false;
    if (d->ly != 0 && (d->ly < 2 * d->ny - 1 || d->ly > 256 || !is_smooth(d->ly))) return false;
    const int lx = d->lx ? d->lx : smooth_size_at_least(2 * d->nx - 1);
    const int ly = d->ly ? d->ly : smooth_size_at_least(2 * d->ny - 1);
    if (d->edge_per_cell < 0 || d->edge_per_cell > 8) return false;
    if (d->edge_per_cell > 0) {  // perimeter layout: exact count, no absent elements
        if ((int64_t)d->n_edge != 2LL * d->edge_per_cell * (d->nx + d->ny)) return false;
        if (d->active)
            for (int k = 0; k < d->nx * d->ny; ++k)
                if (!d->active[k]) return false;
    }
    return lx <= 256 && ly <= 256;
}

static int count_pairs(int lx, int ly, std::vector<int2> *pairs, std::vector<int> *rep) {
    const int F = lx * ly;
    if (rep) rep->assign(F, 0);
    int np = 0;
    for (int ky = 0; ky < ly; ++ky)
        for (int kx = 0; kx < lx; ++kx) {
            const int f = ky * lx + kx;
            const int g = ((ly - ky) % ly) * lx + (lx - kx) % lx;
            if (f <= g) {
                if (pairs) pairs->push_back(make_int2(f, g));
                if (rep) { (*rep)[f] = np; if (g != f) (*rep)[g] = -1 - np; }
                ++np;
            }
        }
    return np;
}

static size_t plan_bytes(int nx, int ny, int b, int E, int lx, int ly, int side_k) {
    const int64_t NT = (int64_t)nx * ny * b;
    const int np = count_pairs(lx, ly, nullptr, nullptr);
    const int64_t ldb = edge_row_stride(NT);
    size_t s = 0;
    s += (size_t)np * b * b * (16 + 8);
    if (side_k > 0)
        s += (size_t)4 * side_k * lx * ly * b * (16 + 8);  // side generator spectra
    else
        s += (size_t)E * ldb * 16 + (size_t)E * edge_row_stride32(NT, E) * 8;
    s += (size_t)E * E * (16 + 8);
    s += (size_t)lx * ly * (sizeof(int) + sizeof(int2)) + (size_t)(lx + ly) * 24 + (size_t)nx * ny + 64;
    return s;
}

}  // namespace ztoep

using namespace ztoep;

extern "C" {

const char *ztoep_version(void) { return "ztoep 0.1 sm_103a"; }

const char *ztoep_status_string(ztoep_status_t s) {
    switch (s) {
        case ZTOEP_OK: return "ok";
        case ZTOEP_ERR_ARG: return "invalid argument";
        case ZTOEP_ERR_NOMEM: return "out of device memory";
        case ZTOEP_ERR_CUDA: return "CUDA error";
        case ZTOEP_ERR_NOCONV: return "not converged";
        case ZTOEP_ERR_TIMEOUT: return "timeout";
        case ZTOEP_ERR_UNSUPPORTED: return "unsupported";
        case ZTOEP_ERR_NONFINITE: return "non-finite value";
    }
    return "unknown status";
}

ztoep_status_t ztoep_default_opts(ztoep_solve_opts_t *o) {
    if (!o) return ZTOEP_ERR_ARG;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-8;
    o->restart = 30;
    o->max_iter = 4000;
    o->max_outer = 100;
    o->prec = ZTOEP_MIXED;
    o->inner_tol = 1e-5;
    o->timeout_ns = 0;
    o->flags = 0;
    return ZTOEP_OK;
}

void ztoep_plan_destroy(ztoep_plan_t p) {
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    if (p->side) cudaStreamSynchronize(p->side);
    free_matvec_ws(p);
    free_solve_ws(p);
    cudaFree(p->pairs); cudaFree(p->rep);
    cudaFree(p->That64); cudaFree(p->That32);
    cudaFree(p->B64); cudaFree(p->B32); cudaFree(p->C64); cudaFree(p->C32);
    cudaFree(p->That32full); cudaFree(p->B32T); cudaFree(p->G64); cudaFree(p->G32);
    cudaFree(p->active);
    cudaFree(p->twx64); cudaFree(p->twy64); cudaFree(p->twx32); cudaFree(p->twy32);
    cudaFree(p->err);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->ev_et) cudaEventDestroy(p->ev_et);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->aux) cudaStreamDestroy(p->aux);
    cudaSetDevice(cur);
    delete p;
}

static ztoep_status_t upload_twiddles(int L, double2 **d64, float2 **d32, size_t *acc, cudaStream_t s) {
    std::vector<double2> h64(L);
    std::vector<float2> h32(L);
    for (int t = 0; t < L; ++t) {
        // exp(-2 pi i t / L), angle reduced to [0, pi/4]-style symmetry by using t/L exactly
        const double a = -2.0 * M_PI * (double)t / (double)L;
        h64[t] = make_double2(std::cos(a), std::sin(a));
        h32[t] = make_float2((float)h64[t].x, (float)h64[t].y);
    }
    ZT_TRY(dalloc((void **)d64, sizeof(double2) * L, acc));
    ZT_TRY(dalloc((void **)d32, sizeof(float2) * L, acc));
    ZT_CUDA(cudaMemcpyAsync(*d64, h64.data(), sizeof(double2) * L, cudaMemcpyHostToDevice, s));
    ZT_CUDA(cudaMemcpyAsync(*d32, h32.data(), sizeof(float2) * L, cudaMemcpyHostToDevice, s));
    return ZTOEP_OK;
}

static ztoep_status_t plan_build(ztoep_plan_t p, const ztoep_desc_t *d, const double2 *T, const double2 *B,
                                 const double2 *C, cudaStream_t s) {
    size_t acc = 0;
    const TuneParams &tp = p->tune;
    p->nx = d->nx; p->ny = d->ny; p->b = d->b; p->E = d->n_edge;
    p->lx = d->lx ? d->lx : smooth_size_at_least(2 * d->nx - 1);
    p->ly = d->ly ? d->ly : smooth_size_at_least(2 * d->ny - 1);
    p->F = p->lx * p->ly;
    p->NT = (int64_t)p->nx * p->ny * p->b;
    p->N = p->NT + p->E;
    p->fx = make_fft1d(p->lx, tp.rad_order[0]);
    p->fy = make_fft1d(p->ly, tp.rad_order[1]);
    ZT_CUDA(cudaGetDevice(&p->device));
    ZT_CUDA(cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device));
    ZT_CUDA(cudaDeviceGetAttribute(&p->l2_bytes, cudaDevAttrL2CacheSize, p->device));
    ZT_CUDA(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    ZT_CUDA(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    ZT_CUDA(cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking));
    ZT_CUDA(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    ZT_CUDA(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    ZT_CUDA(cudaEventCreateWithFlags(&p->ev_et, cudaEventDisableTiming));
    ZT_TRY(dalloc((void **)&p->err, sizeof(int) * 4, &acc));
    ZT_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int) * 4, s));

    // activity mask
    if (d->active) {
        const int nel = p->nx * p->ny;
        bool any_absent = false;
        for (int k = 0; k < nel; ++k) any_absent |= (d->active[k] == 0);
        if (any_absent) {
            p->masked = true;
            ZT_TRY(dalloc((void **)&p->active, nel, &acc));
            ZT_CUDA(cudaMemcpyAsync(p->active, d->active, nel, cudaMemcpyHostToDevice, s));
        }
    }

    // frequency pairs
    std::vector<int2> pairs;
    std::vector<int> rep;
    p->npairs = count_pairs(p->lx, p->ly, &pairs, &rep);
    ZT_TRY(dalloc((void **)&p->pairs, sizeof(int2) * p->npairs, &acc));
    ZT_TRY(dalloc((void **)&p->rep, sizeof(int) * p->F, &acc));
    ZT_CUDA(cudaMemcpyAsync(p->pairs, pairs.data(), sizeof(int2) * p->npairs, cudaMemcpyHostToDevice, s));
    ZT_CUDA(cudaMemcpyAsync(p->rep, rep.data(), sizeof(int) * p->F, cudaMemcpyHostToDevice, s));
    ZT_TRY(upload_twiddles(p->lx, &p->twx64, &p->twx32, &acc, s));
    ZT_TRY(upload_twiddles(p->ly, &p->twy64, &p->twy32, &acc, s));

    // transformed generating blocks
    const int bb = p->b * p->b;
    ZT_TRY(dalloc((void **)&p->That64, sizeof(double2) * (size_t)p->npairs * bb, &acc));
    ZT_TRY(dalloc((void **)&p->That32, sizeof(float2) * (size_t)p->npairs * bb, &acc));
    {
        double2 *P1 = nullptr;
        ZT_TRY(dalloc((void **)&P1, sizeof(double2) * (size_t)(2 * p->ny - 1) * p->lx * bb, nullptr));
        const int libx = pick_lib(p->lx, bb, sizeof(double2), 64 * 1024, 32);
        const int ibx = 1 << libx;
        dim3 gx((bb + ibx - 1) / ibx, 2 * p->ny - 1, 1);
        ztoep_status_t st = launch_fft_pass<double>(p->fx, p->twx64, libx, false, gx,
                                                    LdPlanX{T, p->nx, p->lx, bb, ibx},
                                                    StPlanX{P1, p->lx, bb, ibx}, s);
        if (st == ZTOEP_OK) {
            const int liby = pick_lib(p->ly, bb, sizeof(double2), 64 * 1024, 32);
            const int iby = 1 << liby;
            dim3 gy((bb + iby - 1) / iby, p->lx, 1);
            st = launch_fft_pass<double>(p->fy, p->twy64, liby, false, gy,
                                         LdPlanY{P1, p->ny, p->ly, p->lx, bb, iby},
                                         StPlanY{p->rep, p->That64, p->That32, p->lx, bb, iby}, s);
        }
        cudaStreamSynchronize(s);
        cudaFree(P1);
        ZT_TRY(st);
    }

    // edge coupling blocks
    if (p->E > 0 && d->edge_per_cell > 0) {  // side generators instead of B
        p->side_k = d->edge_per_cell;
        ZT_TRY(sides_build(p, B, s, &acc));
        ZT_TRY(dalloc((void **)&p->C64, sizeof(double2) * (size_t)p->E * p->E, &acc));
        ZT_TRY(dalloc((void **)&p->C32, sizeof(float2) * (size_t)p->E * p->E, &acc));
        ZT_CUDA(cudaMemcpyAsync(p->C64, C, sizeof(double2) * (size_t)p->E * p->E, cudaMemcpyDeviceToDevice, s));
        ZT_TRY(launch_c128_to_c64(p->C64, p->C32, (int64_t)p->E * p->E, s));
    } else if (p->E > 0) {
        const int64_t ldb = edge_row_stride(p->NT);
        ZT_TRY(dalloc((void **)&p->B64, sizeof(double2) * (size_t)p->E * ldb, &acc));
        ZT_TRY(dalloc((void **)&p->B32, sizeof(float2) * (size_t)p->E * edge_row_stride32(p->NT, p->E), &acc));
        ZT_TRY(dalloc((void **)&p->C64, sizeof(double2) * (size_t)p->E * p->E, &acc));
        ZT_TRY(dalloc((void **)&p->C32, sizeof(float2) * (size_t)p->E * p->E, &acc));
        ZT_CUDA(cudaMemsetAsync(p->B64, 0, sizeof(double2) * (size_t)p->E * ldb, s));
        ZT_CUDA(cudaMemcpy2DAsync(p->B64, sizeof(double2) * ldb, B, sizeof(double2) * p->NT,
                                  sizeof(double2) * p->NT, p->E, cudaMemcpyDeviceToDevice, s));
        if (p->masked) {
            KScope ks(K_MISC, s);
            k_zero_columns<<<1024, 256, 0, s>>>(p->B64, ldb, p->E, p->active, p->nx * p->ny, p->b);
            ZT_CUDA(cudaGetLastError());
        }
        ZT_CUDA(cudaMemcpyAsync(p->C64, C, sizeof(double2) * (size_t)p->E * p->E, cudaMemcpyDeviceToDevice, s));
        ZT_TRY(launch_c128_to_c64(p->C64, p->C32, (int64_t)p->E * p->E, s));
        ZT_TRY(pack_bc32(p, s));
    }
    p->resident = acc;
    return ZTOEP_OK;
}

}  // extern "C"

namespace ztoep {
ztoep_status_t plan_create(const ztoep_desc_t *d, const void *T, const void *B, const void *C, cudaStream_t s,
                           const TuneParams &tp, ztoep_plan_t *out) {
    if (!out) return ZTOEP_ERR_ARG;
    *out = nullptr;
    if (!valid_desc(d) || !T) return ZTOEP_ERR_ARG;
    if (d->n_edge > 0 && (!B || !C)) return ZTOEP_ERR_ARG;
    ztoep_plan_t p = new (std::nothrow) ztoep_plan_s();
    if (!p) return ZTOEP_ERR_NOMEM;
    p->tune = tp;
    ztoep_status_t st = plan_build(p, d, (const double2 *)T, (const double2 *)B, (const double2 *)C, s);
    if (st != ZTOEP_OK) {
        ztoep_plan_destroy(p);
        return st;
    }
    *out = p;
    return ZTOEP_OK;
}
}  // namespace ztoep

extern "C" {

ztoep_status_t ztoep_plan(const ztoep_desc_t *d, const void *T, const void *B, const void *C, void *stream,
                          ztoep_plan_t *out) {
    return plan_create(d, T, B, C, (cudaStream_t)stream, TuneParams{}, out);
}

ztoep_status_t ztoep_plan_get_info(ztoep_plan_t p, ztoep_plan_info_t *info) {
    if (!p || !info) return ZTOEP_ERR_ARG;
    info->nx = p->nx; info->ny = p->ny; info->b = p->b; info->n_edge = p->E;
    info->lx = p->lx; info->ly = p->ly;
    info->n_toep = p->NT; info->n = p->N;
    info->n_pairs = p->npairs;
    info->resident_bytes = p->resident + p->tc_bytes + p->ws32.bytes + p->ws64.bytes + p->sws.bytes;
    info->dense_bytes = (size_t)p->N * (size_t)p->N * 16;
    return ZTOEP_OK;
}

size_t ztoep_footprint(const ztoep_desc_t *d, int32_t max_nrhs, int32_t restart) {
    if (!valid_desc(d) || max_nrhs < 1 || restart < 1) return 0;
    const int lx = d->lx ? d->lx : smooth_size_at_least(2 * d->nx - 1);
    const int ly = d->ly ? d->ly : smooth_size_at_least(2 * d->ny - 1);
    const int64_t NT = (int64_t)d->nx * d->ny * d->b, N = NT + d->n_edge;
    size_t s = plan_bytes(d->nx, d->ny, d->b, d->n_edge, lx, ly, d->edge_per_cell);
    // matvec workspaces (FP32 and FP64): in/out copies, x-pass lines, spectrum, edge partials
    const size_t per_rhs = (size_t)(2 * N + (int64_t)d->ny * lx * d->b + (int64_t)lx * ly * d->b + 8 * NT) * 24;
    s += per_rhs * max_nrhs;
    // Krylov basis and vectors (FP64)
    s += (size_t)max_nrhs * N * 16 * (restart + 8);
    // tensor-core operands for 16+ RHS: full FP32 spectrum, transposed B (dense B only), product output
    if (max_nrhs >= kTcMinRhs)
        s += (size_t)lx * ly * d->b * d->b * 8 + (d->edge_per_cell ? 0 : (size_t)NT * d->n_edge * 8) +
             (size_t)lx * ly * d->b * max_nrhs * 8;
    return s;
}

ztoep_status_t ztoep_matvec(ztoep_plan_t p, int32_t prec, int32_t nrhs, const void *X, void *Y, void *stream) {
    if (!p || !X || !Y || nrhs < 1) return ZTOEP_ERR_ARG;
    const size_t vbytes = sizeof(double2) * (size_t)nrhs * p->N;
    if (bytes_overlap(X, vbytes, Y, vbytes)) return ZTOEP_ERR_ARG;
    if (prec != ZTOEP_FP64 && prec != ZTOEP_MIXED) return ZTOEP_ERR_ARG;
    std::lock_guard<std::mutex> lk(p->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == ZTOEP_FP64)
        return run_matvec<double>(p, nrhs, (const double2 *)X, (double2 *)Y, s);
    ZT_TRY(ensure_ws<float>(p, nrhs));
    ZT_TRY(ensure_tensor_data(p, nrhs, s));
    float2 *xin = (float2 *)p->ws32.xin, *yout = (float2 *)p->ws32.yout;
    ZT_TRY(launch_c128_to_c64((const double2 *)X, xin, (int64_t)nrhs * p->N, s));
    ZT_TRY(run_matvec<float>(p, nrhs, xin, yout, s));
    return launch_c64_to_c128(yout, (double2 *)Y, (int64_t)nrhs * p->N, s);
}

ztoep_status_t ztoep_forward_spectrum(ztoep_plan_t p, int32_t prec, int32_t nrhs, const void *X, void *Xhat,
                                      void *stream) {
    if (!p || !X || !Xhat || nrhs < 1) return ZTOEP_ERR_ARG;
    if (prec != ZTOEP_FP64 && prec != ZTOEP_MIXED) return ZTOEP_ERR_ARG;
    std::lock_guard<std::mutex> lk(p->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == ZTOEP_FP64)
        return run_forward_spectrum<double>(p, nrhs, (const double2 *)X, (double2 *)Xhat, s);
    ZT_TRY(ensure_ws<float>(p, nrhs));
    float2 *xin = (float2 *)p->ws32.xin;
    float2 *xh = (float2 *)p->ws32.Xh;
    ZT_TRY(launch_c128_to_c64((const double2 *)X, xin, (int64_t)nrhs * p->N, s));
    ZT_TRY(run_forward_spectrum<float>(p, nrhs, xin, xh, s));
    return launch_c64_to_c128(xh, (double2 *)Xhat, (int64_t)p->F * nrhs * p->b, s);
}

ztoep_status_t ztoep_plan_spectrum(ztoep_plan_t p, void *That, void *stream) {
    if (!p || !That) return ZTOEP_ERR_ARG;
    KScope ks(K_MISC, (cudaStream_t)stream);
    k_expand_spectrum<<<1024, 256, 0, (cudaStream_t)stream>>>(p->That64, p->rep, (double2 *)That, p->F, p->b);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

}  // extern "C"
