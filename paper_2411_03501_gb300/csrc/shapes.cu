// shapes.cu -- implicit surfaces on the device (Sec. III-C: signed distance
// primitives; Sec. III-D: calculus on implicit functions), for building
// targets and initial fields without a host round trip.
//
// One thread per node (grid-stride), coordinates lo + i * dx per axis as the
// stage kernels use them, in the field's precision (FP64 arithmetic for FP32
// fields would run on GB300's slow FP64 pipe).  Primitives measure distance in the non-ignored
// dimensions only (ignoring dimensions turns a sphere into a cylinder, a box
// into a slab); periodic axes are not wrapped.
#include <cmath>

#include "../../include/lsp.h"
#include "launch.h"
#include "stencil.cuh"

namespace lsp {

template <typename R>
__device__ __forceinline__ R shape_value(const ShapeGeom& g, const ShapeArgs& s, const R* x)
{
    if (s.kind == SHAPE_SPHERE) {  // |x - c| - r
        R q = R(0);
        for (int k = 0; k < g.ndim; ++k)
            if (!((s.ignore >> k) & 1u)) q += (x[k] - R(s.c[k])) * (x[k] - R(s.c[k]));
        return rsqrt_(q) - R(s.r);
    }
    if (s.kind == SHAPE_BOX) {  // exact signed distance to [c, d]
        R out2 = R(0), in = R(-INFINITY);
        for (int k = 0; k < g.ndim; ++k) {
            if ((s.ignore >> k) & 1u) continue;
            const R e = rmax(R(s.c[k]) - x[k], x[k] - R(s.d[k]));  // > 0 outside this slab
            if (e > R(0)) out2 += e * e;
            in = rmax(in, e);
        }
        return out2 > R(0) ? rsqrt_(out2) : in;
    }
    if (s.kind == SHAPE_QUADRIC) {  // sum_k w_k (x_k - c_k)^2 - offset
        R q = R(0);
        for (int k = 0; k < g.ndim; ++k)
            if (!((s.ignore >> k) & 1u)) q += R(s.d[k]) * (x[k] - R(s.c[k])) * (x[k] - R(s.c[k]));
        return q - R(s.r);
    }
    // half space {n . (x - p) <= 0}: signed distance n . (x - p) / |n|
    R q = R(0), nn = R(0);
    for (int k = 0; k < g.ndim; ++k)
        if (!((s.ignore >> k) & 1u)) {
            q += R(s.d[k]) * (x[k] - R(s.c[k]));
            nn += R(s.d[k]) * R(s.d[k]);
        }
    return q / rsqrt_(nn);
}

template <typename R>
__global__ void __launch_bounds__(256) shape_kernel(ShapeGeom g, ShapeArgs s, R* out)
{
    // 32-bit index arithmetic (the host checks npts < 2^31): 64-bit division
    // per node would dominate these memory-bound kernels
    const unsigned npts = (unsigned)g.npts;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += gridDim.x * blockDim.x) {
        R x[LSP_MAXD];
        unsigned r = i;
        for (int k = g.ndim - 1; k >= 0; --k) {
            const unsigned nk = (unsigned)g.n[k], q = r / nk;
            x[k] = R(g.lo[k]) + R(r - q * nk) * R(g.h[k]);
            r = q;
        }
        out[i] = shape_value<R>(g, s, x);
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
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

cudaError_t launch_shape(const ShapeGeom& g, const ShapeArgs& s, int dtype, void* out,
                         cudaStream_t st)
{
    if (dtype == LSP_F64)
        shape_kernel<double><<<shape_blocks(g.npts), 256, 0, st>>>(g, s, (double*)out);
    else
        shape_kernel<float><<<shape_blocks(g.npts), 256, 0, st>>>(g, s, (float*)out);
    return cudaGetLastError();
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
