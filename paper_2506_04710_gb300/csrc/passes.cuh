// Load/store functors of the FFT passes of the product: each maps (position
// along the transformed axis, channel in the CTA's batch) of the CTA's line
// (blockIdx.y: line, blockIdx.z: RHS, blockIdx.x: channel batch of ib) to
// global memory.  The layouts are those of the pipeline in matvec.cu.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace ztoep {

// ------------------------------------------------------------ FFT functors
// Each maps (position along the transformed axis, channel in the CTA's batch)
// to global memory; ld2/st2 move the channel pair (ch, ch+1) of FP32 passes
// as one 16-byte access when it is aligned (two 8-byte ones otherwise).
__device__ __forceinline__ float4 ld_pair(const float2 *p, bool two) {
    if (!two) return make_float4(p[0].x, p[0].y, 0.f, 0.f);
    if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) return *reinterpret_cast<const float4 *>(p);
    return make_float4(p[0].x, p[0].y, p[1].x, p[1].y);
}
__device__ __forceinline__ void st_pair(float2 *p, bool two, float4 v) {
    if (!two) {
        p[0] = make_float2(v.x, v.y);
    } else if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
        *reinterpret_cast<float4 *>(p) = v;
    } else {
        p[0] = make_float2(v.x, v.y);
        p[1] = make_float2(v.z, v.w);
    }
}
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

template <typename R> struct LdXFwd {  // x[r][(n*nx+m)*b+i], masked, zero beyond nx
    const cplx_t<R> *x; const uint8_t *active; int nx, b, ib; int64_t N;
    __device__ cplx_t<R> operator()(int m, int ch) const {
        const int n = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (m >= nx || i >= b) return czero<cplx_t<R>>();
        const int el = n * nx + m;
        if (active && !active[el]) return czero<cplx_t<R>>();
        return x[(int64_t)r * N + (int64_t)el * b + i];
    }
    __device__ float4 ld2(int m, int ch) const {
        const int n = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (m >= nx || i >= b) return zero4();
        const int el = n * nx + m;
        if (active && !active[el]) return zero4();
        return ld_pair(x + (int64_t)r * N + (int64_t)el * b + i, i + 1 < b);
    }
};
template <typename R> struct StX1 {  // X1[r][n][kx][i]
    cplx_t<R> *X1; int ny, lx, b, ib;
    __device__ void operator()(int kx, int ch, cplx_t<R> v) const {
        const int n = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (i < b) X1[(((int64_t)r * ny + n) * lx + kx) * b + i] = v;
    }
    __device__ void st2(int kx, int ch, float4 v) const {
        const int n = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (i < b) st_pair(X1 + (((int64_t)r * ny + n) * lx + kx) * b + i, i + 1 < b, v);
    }
};
template <typename R> struct LdX1 {  // X1[r][n][kx][i], zero beyond ny; grid.y = kx
    const cplx_t<R> *X1; int ny, lx, b, ib;
    __device__ cplx_t<R> operator()(int n, int ch) const {
        const int kx = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (n >= ny || i >= b) return czero<cplx_t<R>>();
        return X1[(((int64_t)r * ny + n) * lx + kx) * b + i];
    }
    __device__ float4 ld2(int n, int ch) const {
        const int kx = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (n >= ny || i >= b) return zero4();
        return ld_pair(X1 + (((int64_t)r * ny + n) * lx + kx) * b + i, i + 1 < b);
    }
};
template <typename R> struct StXh {  // Xh[f][r][i]
    cplx_t<R> *Xh; int lx, b, ib, nrhs;
    __device__ void operator()(int ky, int ch, cplx_t<R> v) const {
        const int kx = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (i < b) Xh[(((int64_t)ky * lx + kx) * nrhs + r) * b + i] = v;
    }
    __device__ void st2(int ky, int ch, float4 v) const {
        const int kx = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (i < b) st_pair(Xh + (((int64_t)ky * lx + kx) * nrhs + r) * b + i, i + 1 < b, v);
    }
};
template <typename R> struct LdXh {
    const cplx_t<R> *Xh; int lx, b, ib, nrhs;
    __device__ cplx_t<R> operator()(int ky, int ch) const {
        const int kx = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (i >= b) return czero<cplx_t<R>>();
        return Xh[(((int64_t)ky * lx + kx) * nrhs + r) * b + i];
    }
    __device__ float4 ld2(int ky, int ch) const {
        const int kx = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (i >= b) return zero4();
        return ld_pair(Xh + (((int64_t)ky * lx + kx) * nrhs + r) * b + i, i + 1 < b);
    }
};
template <typename R> struct StY1 {  // crop n < ny
    cplx_t<R> *X1; int ny, lx, b, ib;
    __device__ void operator()(int n, int ch, cplx_t<R> v) const {
        const int kx = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (n < ny && i < b) X1[(((int64_t)r * ny + n) * lx + kx) * b + i] = v;
    }
    __device__ void st2(int n, int ch, float4 v) const {
        const int kx = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (n < ny && i < b) st_pair(X1 + (((int64_t)r * ny + n) * lx + kx) * b + i, i + 1 < b, v);
    }
};
template <typename R> struct LdY1 {  // grid.y = n
    const cplx_t<R> *X1; int ny, lx, b, ib;
    __device__ cplx_t<R> operator()(int kx, int ch) const {
        const int n = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (i >= b) return czero<cplx_t<R>>();
        return X1[(((int64_t)r * ny + n) * lx + kx) * b + i];
    }
    __device__ float4 ld2(int kx, int ch) const {
        const int n = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (i >= b) return zero4();
        return ld_pair(X1 + (((int64_t)r * ny + n) * lx + kx) * b + i, i + 1 < b);
    }
};
template <typename R> struct StYOut {  // crop m < nx, scale, + B^T x_E partials, identity on absent elements
    cplx_t<R> *y; const cplx_t<R> *xin; const cplx_t<R> *ET; const uint8_t *active;
    int nx, b, ib, nrhs, nsplit; int64_t N, NT; R scale;
    __device__ void operator()(int m, int ch, cplx_t<R> v) const {
        const int n = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (m >= nx || i >= b) return;
        const int el = n * nx + m;
        const int64_t t = (int64_t)el * b + i;
        cplx_t<R> out;
        if (active && !active[el]) {
            out = xin[(int64_t)r * N + t];
        } else {
            out = cscale(v, scale);
            for (int s = 0; s < nsplit; ++s) out = out + ET[((int64_t)s * nrhs + r) * NT + t];
        }
        y[(int64_t)r * N + t] = out;
    }
    __device__ void st2(int m, int ch, float4 v) const {
        const int n = blockIdx.y, r = blockIdx.z, i = blockIdx.x * ib + ch;
        if (m >= nx || i >= b) return;
        const int el = n * nx + m;
        const int64_t t = (int64_t)el * b + i;
        const bool two = i + 1 < b;
        float4 out;
        if (active && !active[el]) {
            out = ld_pair(xin + (int64_t)r * N + t, two);
        } else {
            out = make_float4(v.x * scale, v.y * scale, v.z * scale, v.w * scale);
            for (int s = 0; s < nsplit; ++s) {
                const float4 e = ld_pair(ET + ((int64_t)s * nrhs + r) * NT + t, two);
                out = make_float4(out.x + e.x, out.y + e.y, out.z + e.z, out.w + e.w);
            }
        }
        st_pair(y + (int64_t)r * N + t, two, out);
    }
};

}  // namespace ztoep
