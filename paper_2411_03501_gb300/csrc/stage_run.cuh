// stage_run.cuh -- the fused Runge-Kutta stage (Sec. V-A) for the ENO2 and
// ENO3 schemes (Sec. IV-B) on 3-D and 4-D FP32 grids, with every one-sided
// derivative taken from a cell-face evaluation that serves both of its
// nodes.
//
// Same computation as tiled_stage_body<.., ENO2/ENO3, ..> (stage_tiled.cuh):
// ghost cells (Sec. III-B), one-sided ENO derivatives along every axis, the
// LF numerical Hamiltonian with global-LF dissipation (Sec. IV-D), the RK
// combination and the min with the target (Sec. VI-A).  Organised for the
// instruction issue rate, which bounds these schemes on GB300:
//  - ENO selections are made once per cell face.  The ENO polynomial of the
//    right-biased derivative at node j and of the left-biased one at node
//    j+1 starts from the same interval [x_j, x_j+1] (k = j for both), so the
//    second-difference choice, the base index k* and the third-difference
//    choice are the same; only the evaluation point differs (Eqs. 11-14):
//      p+_j    = d - c/2 + cs f+/6,   p-_{j+1} = d + c/2 + cs f-/6,
//      (f+, f-) = (-1, 2) if the left second difference was taken, else (2, -1),
//    with d = u_{j+1} - u_j, c the chosen second difference and cs the
//    chosen third difference (all unscaled; 1/dx is applied once per axis).
//    With M_j the smaller in magnitude of T_{j-1/2}, T_{j+1/2} (ties to the
//    left, the <= of Eq. 13), cs = M_j when the left second difference is
//    taken and M_{j+1} otherwise, so M is formed once per node.
//  - Each thread owns a run of R = 4 (or 2) consecutive nodes of the fastest
//    axis B: the run's faces along B are evaluated once (R + 1 faces);
//    along the marching axis S a register pipeline carries the differences,
//    the M values and the left-biased derivative of the next plane, so one
//    face per node and plane is evaluated; the tile axis A and, in 4-D, the
//    slowest axis (a grid dimension) take both faces per node.
//  - The plane tile with its G-cell halo is staged in shared memory by
//    per-element asynchronous copies (cp.async), double-buffered; ghost
//    values of periodic axes are copies of the wrapped nodes, those of
//    extrapolated axes are formed from the staged nodes; the run's B window
//    and its A columns are read with R-float vector loads (row pitch and run
//    origin are multiples of R floats).
// Branch-free selections (selects on the comparisons), explicit FMAs.
#pragma once
#include "stage_tiled.cuh"

namespace lsp {

// The marching axis' register pipeline for one node column.  ENO3 carries,
// before plane s: u_{s+2}, d_{s+1/2}, d_{s+3/2}, S_s, S_{s+1}, T_{s+1/2},
// M_s and dx p-_s; ENO2 carries u_{s+1}, d_{s+1/2}, S_s and dx p-_s.
template <int SCHEME>
struct MarchState {
    float u, dA, dB, S0, S1, T1, M0, pm;
};

// Initialise from the window w[k] = u_{s0-G+k}, k = 0..2G-1.
template <int SCHEME>
__device__ __forceinline__ void march_init(const float* w, MarchState<SCHEME>& m)
{
    if constexpr (SCHEME == ENO2) {  // w = u_{s0-2 .. s0+1}
        const float da = w[1] - w[0], db = w[2] - w[1], dc = w[3] - w[2];
        const float Sa = db - da, Sb = dc - db;  // S_{s0-1}, S_{s0}
        float pp_unused;
        eno2_face(db, Sa, Sb, pp_unused, m.pm);  // face s0 - 1/2
        m.u = w[3];
        m.dA = dc;
        m.S0 = Sb;
    } else {  // w = u_{s0-3 .. s0+2}
        float d[5], S[4], T[3];
#pragma unroll
        for (int k = 0; k < 5; ++k) d[k] = w[k + 1] - w[k];  // faces s0-5/2 .. s0+3/2
#pragma unroll
        for (int k = 0; k < 4; ++k) S[k] = d[k + 1] - d[k];  // nodes s0-2 .. s0+1
#pragma unroll
        for (int k = 0; k < 3; ++k) T[k] = S[k + 1] - S[k];  // faces s0-3/2 .. s0+1/2
        const float Mm = eno_smaller(T[0], T[1]), M0 = eno_smaller(T[1], T[2]);
        float pp_unused;
        eno3_face(d[2], S[1], S[2], Mm, M0, pp_unused, m.pm);  // face s0 - 1/2
        m.u = w[5];
        m.dA = d[3];
        m.dB = d[4];
        m.S0 = S[2];
        m.S1 = S[3];
        m.T1 = T[2];
        m.M0 = M0;
    }
}

// Plane s: take the lead value u_{s+G}, return dx p-_s and dx p+_s and
// advance the pipeline to plane s+1.
template <int SCHEME>
__device__ __forceinline__ void march_step(MarchState<SCHEME>& m, float lead, float& pm, float& pp)
{
    pm = m.pm;
    if constexpr (SCHEME == ENO2) {
        const float dB = lead - m.u;  // d_{s+3/2}
        const float S1 = dB - m.dA;   // S_{s+1}
        float pnext;
        eno2_face(m.dA, m.S0, S1, pp, pnext);  // face s + 1/2
        m.u = lead;
        m.dA = dB;
        m.S0 = S1;
        m.pm = pnext;
    } else {
        const float dC = lead - m.u;  // d_{s+5/2}
        const float S2 = dC - m.dB;   // S_{s+2}
        const float T2 = S2 - m.S1;   // T_{s+3/2}
        const float M1 = eno_smaller(m.T1, T2);  // M_{s+1}
        float pnext;
        eno3_face(m.dA, m.S0, m.S1, m.M0, M1, pp, pnext);  // face s + 1/2
        m.u = lead;
        m.dA = m.dB;
        m.dB = dC;
        m.S0 = m.S1;
        m.S1 = S2;
        m.T1 = T2;
        m.M0 = M1;
        m.pm = pnext;
    }
}

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gsrc)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Shared-memory layout of one staged plane (floats):
//  - the haloed tile: rows r = 0..TA+2G-1 hold axis-A index a0 - G + r,
//    columns c hold axis-B index b0 - 4 + c (c = 4 - G .. 4 + TB + G - 1
//    staged), row pitch kPitch = R TBT + 8, so the run of thread tx (nodes
//    b0 + R tx .. + R-1) starts at column 4 + R tx, aligned to R floats;
//  - per tile row, the per-node rows of TB values: in 4-D the 2G planes of
//    the slowest axis' window (offsets -G..-1, 1..G), then the march's lead
//    values u_{s+G}, phi^n and the target.
// Every value a plane's computation reads is copied in asynchronously one
// plane ahead, so the computation itself reads shared memory only.
template <int R, int TBT>
struct RunLayout {
    static constexpr int TB = R * TBT;
    static constexpr int kPitch = TB + 8;
};

// Floats of one plane buffer for ta rows.
template <int NDIM, int SCHEME, int R, int TBT>
__host__ __device__ inline int run_plane_floats(int ta)
{
    constexpr int G = ghost_width(SCHEME);
    constexpr int TB = RunLayout<R, TBT>::TB, P = RunLayout<R, TBT>::kPitch;
    return (ta + 2 * G) * P + ((NDIM == 4 ? 2 * G : 0) + 3) * ta * TB;
}

// R consecutive floats from shared memory aligned to R floats.
template <int R>
__device__ __forceinline__ void ldv(const float* p, float* v)
{
    if constexpr (R == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else {
        static_assert(R == 2, "runs of 2 or 4 nodes");
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x;
        v[1] = t.y;
    }
}

// One CTA's share of a stage.  Block (TBT, TA): thread (tx, ty) owns nodes
// (ia = a0 + ty, ib = b0 + R tx .. b0 + R tx + R-1) of every plane s of
// chunk `chunk` along S, at index `outer` of axis 0 in 4-D.
template <int NDIM, int SCHEME, int DYN, int R, int TBT>
__device__ __forceinline__ void run_stage_body(const StageArgs<float>& a, int bx, int by, int chunk,
                                               int outer, int ch, float* smem)
{
    static_assert(NDIM == 3 || NDIM == 4, "3-D and 4-D grids");
    constexpr int G = ghost_width(SCHEME);
    constexpr int AS = NDIM - 3, AA = NDIM - 2, AB = NDIM - 1;
    constexpr int TB = RunLayout<R, TBT>::TB, P = RunLayout<R, TBT>::kPitch;
    constexpr int WST = TB + 2 * G;            // staged columns per row
    constexpr int KC = (WST + TBT - 1) / TBT;  // staged columns per thread and row
    constexpr int NX = NDIM == 4 ? 2 * G : 0;  // planes of the slowest axis' window
    const int TA = blockDim.y;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int H = TA + 2 * G;
    const int nB = a.n[AB], nA = a.n[AA], nS = a.n[AS];
    const int sA = a.stride[AA], sS = a.stride[AS];
    const int b0 = bx * TB, a0 = by * TA;
    const int ib0 = b0 + R * tx, ia = a0 + ty;
    const int base_outer = NDIM == 4 ? outer * a.stride[0] : 0;
    const int s_begin = chunk * ch, s_end = min(s_begin + ch, nS);
    // block-uniform: the tile's nodes are all inside the grid (no partial
    // runs or rows)
    const bool full = b0 + TB <= nB && a0 + TA <= nA;
    // block-uniform: the haloed tile is inside the grid (no ghost values)
    const bool inner = a0 - G >= 0 && a0 + TA + G <= nA && b0 - G >= 0 && b0 + TB + G <= nB;
    // buffer layout (floats): the haloed tile, then per tile row ty the
    // NX + 3 per-node rows (window planes of axis 0, lead, phi^n, target) of
    // TB values each, so that every per-node row of a thread is at an
    // immediate offset from one address
    constexpr int NQ = NX + 3, QL = NX, QN = NX + 1, QG = NX + 2;
    const int bufsz = H * P + TA * NQ * TB;
    const int own = H * P + ty * NQ * TB + R * tx;  // this thread's run, row q = 0
    const bool perA = a.periodic[AA], perB = a.periodic[AB], perS = a.periodic[AS];
    // block-uniform: extrapolated ghost cells of the haloed tile to fill
    const bool ghostA = !perA && (a0 - G < 0 || a0 + TA + G > nA);
    const bool ghostB = !perB && (b0 - G < 0 || b0 + TB + G > nB);
    const int tid = ty * TBT + tx, nthr = TBT * TA;
    // Fill the extrapolated ghost cells of a staged plane from its nodes
    // (linear extrapolation from the two nodes at the edge, Sec. III-B):
    // columns of axis B in rows inside axis A, rows of axis A in columns
    // inside axis B (corners are never read).
    auto fill_ghosts = [&](float* buf) {
        if (ghostB) {
            for (int e = tid; e < H * 2 * G; e += nthr) {
                const int r = e / (2 * G), g = e - r * (2 * G);
                const int ja = a0 - G + r;
                if (ja < 0 || ja >= nA) continue;
                float* row = buf + r * P + 4 - b0;  // row[jb] = value at column jb
                if (g < G) {  // left edge: jb = -1 .. -G
                    const int jb = -1 - g;
                    if (b0 - G <= jb) row[jb] = fmaf(float(-jb), row[0] - row[1], row[0]);
                } else {  // right edge: jb = nB .. nB + G - 1
                    const int jb = nB + g - G;
                    if (jb < b0 + TB + G) {
                        const float un = row[nB - 1];
                        row[jb] = fmaf(float(jb - nB + 1), un - row[nB - 2], un);
                    }
                }
            }
        }
        if (ghostA) {
            for (int e = tid; e < 2 * G * WST; e += nthr) {
                const int g = e / WST, c = e - g * WST;
                const int jb = b0 - G + c;
                if (jb < 0 || jb >= nB) continue;
                float* col = buf + (G - a0) * P + 4 - b0 + jb;  // col[ja * P] = value at row ja
                if (g < G) {
                    const int ja = -1 - g;
                    if (a0 - G <= ja) col[ja * P] = fmaf(float(-ja), col[0] - col[P], col[0]);
                } else {
                    const int ja = nA + g - G;
                    if (ja < a0 + TA + G) {
                        const float un = col[(nA - 1) * P];
                        col[ja * P] = fmaf(float(ja - nA + 1), un - col[(nA - 2) * P], un);
                    }
                }
            }
        }
    };

    const float dt = a.dt_from_ctl ? float(a.ctl->dt) : a.dt;
    const float cl = a.c_l * dt;
    float hs[NDIM], ha[NDIM];  // 1/(2 dx_k) and alpha_k/(2 dx_k)
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        const float al = a.alpha_from_ctl
                             ? float(__longlong_as_double((long long)a.ctl->alpha_bits[k]))
                             : a.alpha[k];
        hs[k] = 0.5f * a.inv_dx[k];
        ha[k] = al * hs[k];
    }

    // coordinates fixed for this thread; theta (axis 2) is axis B in 3-D and
    // axis A in 4-D
    float xo = 0.0f, xa, xb[R];
    if constexpr (NDIM == 4) xo = fmaf(float(outer), a.h[0], a.lo[0]);
    xa = fmaf(float(ia), a.h[AA], a.lo[AA]);
#pragma unroll
    for (int r = 0; r < R; ++r) xb[r] = fmaf(float(ib0 + r), a.h[AB], a.lo[AB]);
    constexpr bool kTrig = DYN == AIR3D || DYN == CAR4D || DYN == ROCKETS;
    float sth[R], cth[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        sth[r] = 0.0f;
        cth[r] = 1.0f;
    }
    if constexpr (kTrig) {
        if constexpr (NDIM == 3) {
#pragma unroll
            for (int r = 0; r < R; ++r) sincosf(xb[r], &sth[r], &cth[r]);
        } else {
            sincosf(xa, &sth[0], &cth[0]);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                sth[r] = sth[0];
                cth[r] = cth[0];
            }
        }
    }

    // per-node column offsets (clamped into the grid for partial tiles)
    const int ia_c = min(ia, nA - 1);
    int coff[R];
#pragma unroll
    for (int r = 0; r < R; ++r) coff[r] = base_outer + ia_c * sA + min(ib0 + r, nB - 1);

    // march pipeline initialised from u_{s_begin-G .. s_begin+G-1}
    MarchState<SCHEME> ms[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float w[2 * G];
#pragma unroll
        for (int o = 0; o < 2 * G; ++o)
            w[o] = line_value<float>(a.phi_s + coff[r], s_begin - G + o, nS, sS, a.periodic[AS]);
        march_init<SCHEME>(w, ms[r]);
    }

    // Copy everything plane p's computation reads into `buf`: asynchronous
    // copies where the value is a grid node, plain stores of ghost values
    // (periodic wrap or linear extrapolation, Sec. III-B) elsewhere.
    auto stage = [&](int p, float* buf) {
        const float* plane = a.phi_s + base_outer + p * sS;
        for (int r = ty; r < H; r += TA) {
            const int ja = a0 - G + r;
            float* srow = buf + r * P + (4 - G) + tx;
            const int jb0 = b0 - G + tx;
            if (inner) {
                const float* grow = plane + ja * sA + jb0;
#pragma unroll
                for (int k = 0; k < KC; ++k)
                    if (k < KC - 1 || tx + k * TBT < WST) cp_async4(srow + k * TBT, grow + k * TBT);
                continue;
            }
            // ghost rows / columns of periodic axes are copies of the
            // wrapped nodes; extrapolated ones are filled from shared memory
            // once the plane has arrived (fill_ghosts), corners are never read
            const bool inA = ja >= 0 && ja < nA;
            const int jaw = inA ? ja : (ja < 0 ? ja + nA : ja - nA);
            if (!inA && (!perA || jaw < 0 || jaw >= nA)) continue;
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                if (k == KC - 1 && tx + k * TBT >= WST) break;
                const int jb = jb0 + k * TBT;
                const bool inB = jb >= 0 && jb < nB;
                if (inB) {
                    cp_async4(srow + k * TBT, plane + jaw * sA + jb);
                } else if (inA && perB) {
                    const int jbw = jb < 0 ? jb + nB : jb - nB;
                    if (jbw >= 0 && jbw < nB) cp_async4(srow + k * TBT, plane + ja * sA + jbw);
                }
            }
        }
        // a full run's nodes are consecutive in memory: one address per
        // copy group, the others at immediate offsets
        auto copy_run = [&](float* dst, const float* src0) {
            if (full) {
#pragma unroll
                for (int r = 0; r < R; ++r) cp_async4(dst + r, src0 + r);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) cp_async4(dst + r, src0 + (coff[r] - coff[0]));
            }
        };
        if constexpr (NDIM == 4) {
            const int s0 = a.stride[0], n0 = a.n[0];
            const float* col0 = a.phi_s + (coff[0] - base_outer) + p * sS;
#pragma unroll
            for (int q = 0; q < NX; ++q) {
                const int o = q < G ? q - G : q - G + 1;
                int j = outer + o;
                float* dst = buf + own + q * TB;
                if (j >= 0 && j < n0) {
                    copy_run(dst, col0 + j * s0);
                } else if (a.periodic[0]) {
                    j = j < 0 ? j + n0 : j - n0;
                    copy_run(dst, col0 + j * s0);
                }  // extrapolated: formed from the window at use time
            }
        }
        const int jl = p + G;  // the march's lead value
        if (jl < nS) {
            copy_run(buf + own + QL * TB, a.phi_s + coff[0] + jl * sS);
        } else if (perS) {
            copy_run(buf + own + QL * TB, a.phi_s + coff[0] + (jl - nS) * sS);
        }  // extrapolated: continued from the march pipeline at use time
        if (a.phi_n) copy_run(buf + own + QN * TB, a.phi_n + coff[0] + p * sS);
        if (a.tube) copy_run(buf + own + QG * TB, a.target + coff[0] + p * sS);
        cp_async_commit();
    };

    stage(s_begin, smem);
    bool nonfinite = false;
    for (int s = s_begin; s < s_end; ++s) {
        const float* cur = smem + ((s - s_begin) & 1) * bufsz;
        cp_async_wait_all();
        __syncthreads();  // plane s staged; the other buffer is free
        if (ghostA || ghostB) {  // block-uniform
            fill_ghosts(const_cast<float*>(cur));
            __syncthreads();
        }
        if (s + 1 < s_end) stage(s + 1, smem + ((s + 1 - s_begin) & 1) * bufsz);

        float pbar[R][NDIM], diss[R];
        // axis B: the run's window from its row, faces shared
        float center[R];
        {
            const float* row = cur + (ty + G) * P + R * tx;
            float w[R + 8];  // columns R tx .. R tx + R + 7
#pragma unroll
            for (int v = 0; v < (R + 8) / R; ++v) ldv<R>(row + v * R, w + v * R);
            // window of the run: columns 4 - G .. 4 + R - 1 + G of w
            float pm[R], pp[R];
            eno_line<SCHEME, R>(w + 4 - G, pm, pp);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                center[r] = w[4 + r];
                pbar[r][AB] = (pp[r] + pm[r]) * hs[AB];
                diss[r] = ha[AB] * (pp[r] - pm[r]);
            }
        }
        // axis A: the run's columns, rows ty .. ty + 2G
        {
            float col[2 * G + 1][R];
#pragma unroll
            for (int o = 0; o <= 2 * G; ++o) ldv<R>(cur + (ty + o) * P + 4 + R * tx, col[o]);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float w[2 * G + 1], pm, pp;
#pragma unroll
                for (int o = 0; o <= 2 * G; ++o) w[o] = col[o][r];
                eno_line<SCHEME, 1>(w, &pm, &pp);
                pbar[r][AA] = (pp + pm) * hs[AA];
                diss[r] = fmaf(ha[AA], pp - pm, diss[r]);
            }
        }
        // axis S: the march pipeline
        {
            float lead[R];
            if (s + G < nS || perS) {
                ldv<R>(cur + own + QL * TB, lead);
            } else {  // beyond the end of an extrapolated axis: the pipeline's
                      // last difference continues (u_{j+1} = u_j + (u_j - u_{j-1}))
#pragma unroll
                for (int r = 0; r < R; ++r)
                    lead[r] = SCHEME == ENO2 ? ms[r].u + ms[r].dA : ms[r].u + ms[r].dB;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float pm, pp;
                march_step<SCHEME>(ms[r], lead[r], pm, pp);
                pbar[r][AS] = (pp + pm) * hs[AS];
                diss[r] = fmaf(ha[AS], pp - pm, diss[r]);
            }
        }
        // axis 0 of a 4-D grid: both faces per node from the staged window
        if constexpr (NDIM == 4) {
            const int n0 = a.n[0];
            const bool in0 = outer >= G && outer + G < n0;  // block-uniform
            float xw[2 * G][R];
#pragma unroll
            for (int q = 0; q < 2 * G; ++q) ldv<R>(cur + own + q * TB, xw[q]);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float w[2 * G + 1], pm, pp;
#pragma unroll
                for (int o = 0; o < G; ++o) {
                    w[o] = xw[o][r];
                    w[G + 1 + o] = xw[G + o][r];
                }
                w[G] = center[r];
                if (!in0 && !a.periodic[0]) {  // block-uniform: extrapolated ghosts
                    // nodes 0, 1 sit at window entries G - outer, G - outer + 1
                    // (outer < G) and nodes n0-1, n0-2 at G + n0-1-outer,
                    // G + n0-2-outer (outer >= n0 - G); selected, not indexed
                    const int lo = outer, hi = n0 - 1 - outer;
                    const float u0 = lo == 0 ? w[G] : (lo == 1 ? w[G - 1] : w[G - 2]);
                    const float u1 = lo == 0 ? w[G + 1] : (lo == 1 ? w[G] : w[G - 1]);
                    const float un = hi == 0 ? w[G] : (hi == 1 ? w[G + 1] : w[G + 2]);
                    const float um = hi == 0 ? w[G - 1] : (hi == 1 ? w[G] : w[G + 1]);
#pragma unroll
                    for (int o = -G; o <= G; ++o) {
                        const int j = outer + o;
                        if (j < 0) w[o + G] = fmaf(float(-j), u0 - u1, u0);
                        else if (j >= n0) w[o + G] = fmaf(float(j - n0 + 1), un - um, un);
                    }
                }
                eno_line<SCHEME, 1>(w, &pm, &pp);
                pbar[r][0] = (pp + pm) * hs[0];
                diss[r] = fmaf(ha[0], pp - pm, diss[r]);
            }
        }
        // Hamiltonian, rate, RK combination, tube; store the active nodes
        float pn[R], tg[R];
        if (a.phi_n) ldv<R>(cur + own + QN * TB, pn);
        if (a.tube) ldv<R>(cur + own + QG * TB, tg);
        const float xs = fmaf(float(s), a.h[AS], a.lo[AS]);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float x[NDIM];
            if constexpr (NDIM == 4) x[0] = xo;
            x[AS] = xs;
            x[AA] = xa;
            x[AB] = xb[r];
            const float Hv = hamiltonian_sc<DYN, NDIM>(x, pbar[r], a.prm, sth[r], cth[r]);
            const float L = diss[r] - Hv;
            float v = fmaf(cl, L, a.c_s * center[r]);
            if (a.phi_n) v = fmaf(a.c_n, pn[r], v);
            if (a.tube) v = fminf(v, tg[r]);
            if (full) {  // consecutive nodes: immediate offsets from one address
                nonfinite |= !isfinite(v);
                a.out[coff[0] + s * sS + r] = v;
            } else if (ia < nA && ib0 + r < nB) {
                nonfinite |= !isfinite(v);
                a.out[coff[r] + s * sS] = v;
            }
        }
    }
    if (nonfinite) atomicOr(&a.ctl->flags, kFlagNonFinite);
}

// Single-problem launch: blockDim = (TBT, ta); gridDim = (ceil(nB / (R TBT)),
// ceil(nA / ta), nchunks * nOuter); dynamic shared memory two plane buffers
// of run_plane_floats(ta) floats.  MINB: CTAs of 256 threads per SM the
// register budget is set for (2: 128 registers per thread, 3: 80).
template <int NDIM, int SCHEME, int DYN, int R, int TBT, int MINB>
__global__ void __launch_bounds__(256, MINB) stage_run_kernel(StageArgs<float> a, int ch, int nchunks)
{
    extern __shared__ float4 run_smem[];
    run_stage_body<NDIM, SCHEME, DYN, R, TBT>(a, blockIdx.x, blockIdx.y, blockIdx.z % nchunks,
                                           blockIdx.z / nchunks, ch,
                                           reinterpret_cast<float*>(run_smem));
}

}  // namespace lsp
