// shapes.cu -- implicit surfaces on the device (Sec. III-C: signed distance
// primitives; Sec. III-D: calculus on implicit functions), for building
// targets and initial fields without a host round trip.
//
// One thread per node (grid-stride), coordinates lo + i * dx per axis as the
// stage kernels use them, in the field's precision (FP64 arithmetic for FP32
// fields would run on GB300's slow FP64 pipe; the shape and grid constants
// are converted once, on the host).  Primitives measure distance in the non-ignored
// dimensions only (ignoring dimensions turns a sphere into a cylinder, a box
// into a slab); periodic axes are not wrapped.
#include <cmath>

#include "../../include/lsp.h"
#include "launch.h"
#include "stencil.cuh"

namespace lsp {

// The kernel's copy of the shape and the grid, in the field precision, with
// the multipliers that divide a node index by each axis length.
template <typename R>
struct ShapeDev {
    R lo[LSP_MAXD], h[LSP_MAXD], c[LSP_MAXD], d[LSP_MAXD], r;
    unsigned n[LSP_MAXD], m[LSP_MAXD];
    int l[LSP_MAXD];
    unsigned ignore, npts;
    int kind;
};

// floor(x / n) for 0 <= x < 2^31 by a multiply-high and a shift (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994:
// l = ceil(log2 n), m = floor(2^32 (2^l - n) / n) + 1, q = (mulhi(m, x) + x) >> l;
// mulhi(m, x) < x, so the sum stays below 2^32)
__device__ __forceinline__ unsigned div_invariant(unsigned x, unsigned m, int l)
{
    return (__umulhi(x, m) + x) >> l;
}

static void division_multiplier(unsigned n, unsigned* m, int* l)
{
    int s = 0;
    while ((1ull << s) < n) ++s;
    *l = s;
    *m = (unsigned)(((((unsigned long long)1 << s) - n) << 32) / n + 1);
}

template <int NDIM, typename R>
__device__ __forceinline__ R shape_value(const ShapeDev<R>& s, const R* x)
{
    if (s.kind == SHAPE_SPHERE) {  // |x - c| - r
        R q = R(0);
#pragma unroll
        for (int k = 0; k < NDIM; ++k)
            if (!((s.ignore >> k) & 1u)) q += (x[k] - s.c[k]) * (x[k] - s.c[k]);
        return real_sqrt(q) - s.r;
    }
    if (s.kind == SHAPE_BOX) {  // exact signed distance to [c, d]
        R out2 = R(0), in = R(-INFINITY);
#pragma unroll
        for (int k = 0; k < NDIM; ++k) {
            if ((s.ignore >> k) & 1u) continue;
            const R e = rmax(s.c[k] - x[k], x[k] - s.d[k]);  // > 0 outside this slab
            if (e > R(0)) out2 += e * e;
            in = rmax(in, e);
        }
        return out2 > R(0) ? real_sqrt(out2) : in;
    }
    if (s.kind == SHAPE_QUADRIC) {  // sum_k w_k (x_k - c_k)^2 - offset
        R q = R(0);
#pragma unroll
        for (int k = 0; k < NDIM; ++k)
            if (!((s.ignore >> k) & 1u)) q += s.d[k] * (x[k] - s.c[k]) * (x[k] - s.c[k]);
        return q - s.r;
    }
    // half space {n . (x - p) <= 0}: signed distance n . (x - p) / |n|
    R q = R(0), nn = R(0);
#pragma unroll
    for (int k = 0; k < NDIM; ++k)
        if (!((s.ignore >> k) & 1u)) {
            q += s.d[k] * (x[k] - s.c[k]);
            nn += s.d[k] * s.d[k];
        }
    return q / real_sqrt(nn);
}

// The coordinates of node i: its index split by the axis lengths (the
// fastest axis last), lo + index * dx per axis as the stage kernels compute
// them.  Dimensions are a template parameter, so the coordinates stay in
// registers; the host checks npts < 2^31 (32-bit index arithmetic).
template <int NDIM, typename R>
__global__ void __launch_bounds__(256) shape_kernel(ShapeDev<R> s, R* out)
{
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < s.npts; i += gridDim.x * blockDim.x) {
        R x[NDIM];
        unsigned r = i;
#pragma unroll
        for (int k = NDIM - 1; k > 0; --k) {
            const unsigned q = div_invariant(r, s.m[k], s.l[k]);
            x[k] = s.lo[k] + R(r - q * s.n[k]) * s.h[k];
            r = q;
        }
        x[0] = s.lo[0] + R(r) * s.h[0];
        out[i] = shape_value<NDIM, R>(s, x);
    }
}

// union min(a, b), intersection max(a, b), complement -a, difference
// max(a, -b) (Sec. III-D)
template <typename R>
__global__ void __launch_bounds__(256) shape_op_kernel(int op, const R* a, const R* b, R* out,
                                                       long long n)
{
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < (unsigned)n;
         i += gridDim.x * blockDim.x) {
        const R u = a[i];
        R v;
        switch (op) {
        case LSP_SHAPE_UNION: v = fmin(u, b[i]); break;
        case LSP_SHAPE_INTERSECT: v = fmax(u, b[i]); break;
        case LSP_SHAPE_COMPLEMENT: v = -u; break;
        default: v = fmax(u, -b[i]); break;
        }
        out[i] = v;
    }
}

static int shape_blocks(long long n)
{
    const long long b = (n + 255) / 256;
    const long long cap = 16LL * sm_count();
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <typename R>
static cudaError_t launch_shape_t(const ShapeGeom& g, const ShapeArgs& s, R* out, cudaStream_t st)
{
    ShapeDev<R> d;
    for (int k = 0; k < LSP_MAXD; ++k) {
        const bool used = k < g.ndim;
        d.lo[k] = used ? R(g.lo[k]) : R(0);
        d.h[k] = used ? R(g.h[k]) : R(0);
        d.c[k] = used ? R(s.c[k]) : R(0);
        d.d[k] = used ? R(s.d[k]) : R(0);
        d.n[k] = used ? (unsigned)g.n[k] : 1u;
        division_multiplier(d.n[k], &d.m[k], &d.l[k]);
    }
    d.r = R(s.r);
    d.ignore = s.ignore;
    d.npts = (unsigned)g.npts;
    d.kind = s.kind;
    const int nb = shape_blocks(g.npts);
    switch (g.ndim) {
    case 1: shape_kernel<1, R><<<nb, 256, 0, st>>>(d, out); break;
    case 2: shape_kernel<2, R><<<nb, 256, 0, st>>>(d, out); break;
    case 3: shape_kernel<3, R><<<nb, 256, 0, st>>>(d, out); break;
    case 4: shape_kernel<4, R><<<nb, 256, 0, st>>>(d, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_shape(const ShapeGeom& g, const ShapeArgs& s, int dtype, void* out,
                         cudaStream_t st)
{
    if (dtype == LSP_F64) return launch_shape_t<double>(g, s, (double*)out, st);
    return launch_shape_t<float>(g, s, (float*)out, st);
}

cudaError_t launch_shape_op(int op, int dtype, const void* a, const void* b, void* out, long long n,
                            cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (dtype == LSP_F64)
        shape_op_kernel<double><<<shape_blocks(n), 256, 0, st>>>(op, (const double*)a,
                                                                 (const double*)b, (double*)out, n);
    else
        shape_op_kernel<float><<<shape_blocks(n), 256, 0, st>>>(op, (const float*)a,
                                                               (const float*)b, (float*)out, n);
    return cudaGetLastError();
}

}  // namespace lsp
