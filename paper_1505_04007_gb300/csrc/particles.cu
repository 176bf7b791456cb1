// particles.cu -- electron push, charge-conserving current deposit, and the
// periodic brick sort that keeps neighbouring electrons in neighbouring
// threads.
//
// Per live electron, one thread in each of two kernels:
//   k_gather_E (beside the H update, which does not touch E): E^n at x^n
//   (staggered trilinear), stored per electron;
//   k_push_deposit (beside the E update, once H^{n+1/2} is final): B^n =
//   mu0 (H^{n-1/2} + H^{n+1/2})/2 at x^n (H^{n-1/2}(x^n) is the value the
//   previous push left in bold), relativistic Boris rotation
//   u^{n-1/2} -> u^{n+1/2}, x^{n+1} = x^n + dt u/gamma,
//   the boundary/metal freeze rule, the Esirkepov current of the move
//   (linear node shapes, 4-node window per axis), and finally
//   bold <- H^{n+1/2}(x^{n+1}) for the next step.
// Positions are kept as (integer cell, offset in [0,1)) so FP32 offsets keep
// full relative precision however large the grid.  The momentum is a
// compensated pair (u + ulo): the Boris step is applied as one increment
// du = 2 h E + u' x s (u' = u- + u- x t), which is computed to full relative
// precision, and folded in with an error-free TwoSum, so per-step momentum
// changes that are ~1e-4 of |u| are not truncated by the FP32 mantissa.
//
// Deposit: a block first finds the bounding box of its electrons' stencil
// windows.  When the box fits in shared memory the block sums all of its
// contributions there (shared-memory atomics) and then adds each non-zero
// edge to J_f once; otherwise every contribution goes to J_f directly.  The
// brick sort (every SORT_EVERY steps, 4x4x4-cell bricks, frozen electrons
// last) keeps a block's electrons in a few bricks, so the box is small.
#include <type_traits>

#include "pic_internal.cuh"

namespace pic {

template <typename T>
__device__ __forceinline__ int wrap_or_clamp(int x, int n, int per) {
    if (per) {
        if (x < 0) x += n;
        else if (x >= n) x -= n;
        return x;
    }
    return x < 0 ? 0 : (x >= n ? n - 1 : x);
}

// Trilinear interpolation at one position on the Yee lattices.  Per axis a
// component lives either on the cell nodes (index c, weight o) or half a
// cell over (index c or c-1, weight o -+ 1/2); the stencil holds both, so
// the six field components share one set of index computations.
template <typename T>
struct Stencil {
    int i0[3][2], i1[3][2];  // [axis][0 unshifted, 1 half-shifted]: lower / upper index
    T w[3][2];               // weight of the upper index
};

template <typename T>
__device__ __forceinline__ void make_stencil(const Grid<T> &g, const int c[3], const T o[3], Stencil<T> &s) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        s.i0[a][0] = c[a];
        s.i1[a][0] = wrap_or_clamp<T>(c[a] + 1, g.n[a], g.per[a]);
        s.w[a][0] = o[a];
        const bool up = o[a] >= T(0.5);
        const int b = up ? c[a] : c[a] - 1;
        s.i0[a][1] = wrap_or_clamp<T>(b, g.n[a], g.per[a]);
        s.i1[a][1] = wrap_or_clamp<T>(b + 1, g.n[a], g.per[a]);
        s.w[a][1] = up ? o[a] - T(0.5) : o[a] + T(0.5);
    }
}

// F on the lattice shifted by half a cell along the axes flagged in STAG
// (bit a): Ex 1, Ey 2, Ez 4; Hx 6, Hy 5, Hz 3.
template <int STAG, typename T>
__device__ __forceinline__ T interp(const T *__restrict__ F, const Grid<T> &g, const Stencil<T> &s) {
    constexpr int sx = STAG & 1, sy = (STAG >> 1) & 1, sz = (STAG >> 2) & 1;
    // 32-bit cell offsets: pic_create takes grids of fewer than 2^32 cells
    const unsigned nx = (unsigned)g.n[0], nxy = (unsigned)g.n[0] * (unsigned)g.n[1];
    const unsigned x0 = (unsigned)s.i0[0][sx], x1 = (unsigned)s.i1[0][sx];
    const unsigned z0 = (unsigned)s.i0[2][sz] * nxy, z1 = (unsigned)s.i1[2][sz] * nxy;
    const unsigned y0 = (unsigned)s.i0[1][sy] * nx, y1 = (unsigned)s.i1[1][sy] * nx;
    const unsigned r00 = z0 + y0, r01 = z0 + y1, r10 = z1 + y0, r11 = z1 + y1;
    const T wx = s.w[0][sx], wy = s.w[1][sy], wz = s.w[2][sz];
    const T ux = T(1) - wx, uy = T(1) - wy, uz = T(1) - wz;
    const T v00 = ux * F[r00 + x0] + wx * F[r00 + x1];
    const T v01 = ux * F[r01 + x0] + wx * F[r01 + x1];
    const T v10 = ux * F[r10 + x0] + wx * F[r10 + x1];
    const T v11 = ux * F[r11 + x0] + wx * F[r11 + x1];
    return uz * (uy * v00 + wy * v01) + wz * (uy * v10 + wy * v11);
}

template <typename T>
__device__ __forceinline__ void interp_H(const Fields<T> &f, const Grid<T> &g, const Stencil<T> &s, T h[3]) {
    h[0] = interp<6>(f.H[0], g, s);
    h[1] = interp<5>(f.H[1], g, s);
    h[2] = interp<3>(f.H[2], g, s);
}

constexpr int PUSH_BLOCK = 256;

__device__ __forceinline__ long long tile_of(const int idx[3], const int nt[3]) {
    return ((long long)(idx[2] / TILE_Z) * nt[1] + idx[1] / TILE_Y) * nt[0] + idx[0] / TILE_X;
}

// The Esirkepov contributions of one electron on a window of WX x WY x WZ
// nodes (2 along an axis no electron of the warp changed cell on, else 3):
// J_c on edge m0 = jscale_c (dS_c[0] + .. + dS_c[m0]) W(m1, m2), with the
// transverse weight W = S0 S0 + (dS S0 + S0 dS)/2 + dS dS/3 written as
// P P + dS dS/12, P = S0 + dS/2.  The cumulative sum is exactly zero past
// the last node with weight, so only edge 0 (and edge 1 when the electron
// changed cell along c) is issued.  Shared path: l0 and st[] index the
// block's node box in acc; direct path: gofs[a][m] is the grid offset of
// window node m along axis a.
//
// FP32: the shared box holds each component in fixed point, as int32 counts
// of a quantum q_c = 1.25 PUSH_BLOCK |jscale_c| / 2^30 (a contribution is at
// most 1.09 |jscale_c| in size and a node takes at most one per electron of
// the block, so a node's sum stays inside int32): native integer atomics in
// shared memory instead of floating-point ones (a dense bunch: 166 -> 136 us
// per push), and the box sums are exact and independent of their order; each
// contribution is rounded to the quantum, 3e-7 |jscale_c|.
constexpr float FIX_Q = 858993459.2f;  // 2^30 / 1.25

template <typename T>
__device__ __forceinline__ float fix_scale(T jscale) {
    return jscale != T(0) ? FIX_Q / (float)(PUSH_BLOCK * fabs(jscale)) : 0.f;
}

template <int WX, int WY, int WZ, typename T>
__device__ __forceinline__ void esirkepov_sites(const T (&P)[3][3], const T (&dS)[3][3], const int (&shv)[3],
                                                const T (&jscale)[3], const float (&fq)[3], bool in_smem, T *acc,
                                                int vol, int l0, const int (&st)[3], T *const (&Jf)[3],
                                                const long long (&gofs)[3][3]) {
    const T twelfth = T(1) / T(12);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
        const int wc = c == 0 ? WX : (c == 1 ? WY : WZ);
        const int w1 = a1 == 0 ? WX : (a1 == 1 ? WY : WZ);
        const int w2 = a2 == 0 ? WX : (a2 == 1 ? WY : WZ);
        const int nedge = shv[c] != 0 ? 2 : 1;
        const T kc[2] = {jscale[c] * dS[c][0], jscale[c] * (dS[c][0] + dS[c][1])};
#pragma unroll
        for (int m2 = 0; m2 < w2; m2++) {
#pragma unroll
            for (int m1 = 0; m1 < w1; m1++) {
                const T tr = P[a1][m1] * P[a2][m2] + twelfth * (dS[a1][m1] * dS[a2][m2]);
                if ((w1 == 3 || w2 == 3) && tr == T(0)) continue;  // a third node with no weight
#pragma unroll
                for (int m0 = 0; m0 < wc - 1; m0++) {
                    if (m0 >= nedge) break;
                    const T v = kc[m0] * tr;
                    if (in_smem) {
                        const int e = c * vol + l0 + m0 * st[c] + m1 * st[a1] + m2 * st[a2];
                        if constexpr (std::is_same<T, float>::value)
                            atomicAdd(reinterpret_cast<int *>(acc) + e, __float2int_rn(v * fq[c]));
                        else
                            atomicAdd(&acc[e], v);
                    } else
                        atomicAdd(&Jf[c][gofs[c][m0] + gofs[a1][m1] + gofs[a2][m2]], v);
                }
            }
        }
    }
}

// GE: E^n is gathered here at x^n (the fused field path, where the push
// runs beside a pass that reads E^n and H^{n+1/2} and writes the other copy
// of the state) rather than read from eg (gathered beside the H update on
// the split path).
template <typename T, bool GE>
__global__ void __launch_bounds__(PUSH_BLOCK, sizeof(T) == 4 ? 4 : 1)
    k_push_deposit(Grid<T> g, Fields<T> f, Particles<T> p, PushParams<T> pp) {
    extern __shared__ __align__(16) unsigned char dep_smem[];
    T *acc = reinterpret_cast<T *>(dep_smem);
    __shared__ int bb_lo[3], bb_hi[3];

    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long step = *f.step;
    bool dep = false;  // this thread deposits a move
    int c0[3], c1[3], c1w[3];
    T o0[3], o1[3];

    if (q < p.n && !p.status[q]) {
        T u[3], ul[3], E[3], B[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            c0[a] = p.cell[a][q]; o0[a] = p.off[a][q]; u[a] = p.u[a][q]; ul[a] = p.ulo[a][q];
            if (!GE) E[a] = p.eg[a][q];
        }
        {
            Stencil<T> st0;
            make_stencil(g, c0, o0, st0);
            T hnew[3], hold3[3];
            interp_H(f, g, st0, hnew);
            if (GE) {
                E[0] = interp<1>(f.E[0], g, st0);
                E[1] = interp<2>(f.E[1], g, st0);
                E[2] = interp<4>(f.E[2], g, st0);
            }
#pragma unroll
            for (int a = 0; a < 3; a++) hold3[a] = p.bold[a][q];
#pragma unroll
            for (int a = 0; a < 3; a++) B[a] = pp.mu0 * T(0.5) * (hold3[a] + hnew[a]);
        }
        // relativistic Boris rotation, as an increment of u
        T um[3], t[3], s[3], up[3], du[3];
#pragma unroll
        for (int a = 0; a < 3; a++) um[a] = (u[a] + ul[a]) + pp.qmdt2 * E[a];
        const T gm = sqrt(T(1) + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]) * pp.inv_c2);
        const T h = pp.qmdt2 / gm;
#pragma unroll
        for (int a = 0; a < 3; a++) t[a] = h * B[a];
        const T t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
        const T sf = T(2) / (T(1) + t2);
#pragma unroll
        for (int a = 0; a < 3; a++) s[a] = sf * t[a];
        up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
        up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
        up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
        du[0] = T(2) * pp.qmdt2 * E[0] + (up[1] * s[2] - up[2] * s[1]);
        du[1] = T(2) * pp.qmdt2 * E[1] + (up[2] * s[0] - up[0] * s[2]);
        du[2] = T(2) * pp.qmdt2 * E[2] + (up[0] * s[1] - up[1] * s[0]);
        T un[3], unl[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            // TwoSum(u, du): exact sum as s + err, then renormalise with the trailing part
            const T sm = u[a] + du[a];
            const T bv = sm - u[a];
            const T err = (u[a] - (sm - bv)) + (du[a] - bv);
            const T lo = ul[a] + err;
            un[a] = sm + lo;
            unl[a] = lo - (un[a] - sm);
        }
        const T gn = sqrt(T(1) + (un[0] * un[0] + un[1] * un[1] + un[2] * un[2]) * pp.inv_c2);
        bool frozen = false;
        if (!isfinite(gn)) {
            atomicOr(pp.err, DEVERR_NONFINITE);
            frozen = true;
        }
        const T ig = T(1) / gn;
        // move in (cell, offset) form; raw cell before periodic wrap for the deposit
#pragma unroll
        for (int a = 0; a < 3; a++) {
            T x = o0[a] + (un[a] + unl[a]) * pp.dtd[a] * ig;
            T fl = floor(x);
            int sh = frozen ? 0 : (int)fl;
            x -= fl;
            if (x >= T(1)) { x -= T(1); sh += 1; }
            if (sh < -1 || sh > 1) { atomicOr(pp.err, DEVERR_JUMP); frozen = true; sh = 0; }
            c1[a] = c0[a] + sh;
            o1[a] = x;
            int w = c1[a];
            if (g.per[a]) {
                if (w < 0) w += g.n[a];
                else if (w >= g.n[a]) w -= g.n[a];
            } else if (w < 2 || w >= g.n[a] - 2) {
                frozen = true;  // within two cells of a non-periodic face
            }
            c1w[a] = w;
        }
        if (!frozen) {
            const long long cell = ((long long)c1w[2] * g.n[1] + c1w[1]) * g.n[0] + c1w[0];
            if (pp.mat_metal[pp.mat[cell]]) frozen = true;  // absorbed by the metal
        }
        if (frozen) {
            p.status[q] = 1;
        } else {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                p.cell[a][q] = c1w[a];
                p.off[a][q] = o1[a];
                p.u[a][q] = un[a];
                p.ulo[a][q] = unl[a];
            }
            {
                Stencil<T> st1;
                make_stencil(g, c1w, o1, st1);
                T hb[3];
                interp_H(f, g, st1, hb);
#pragma unroll
                for (int a = 0; a < 3; a++) p.bold[a][q] = hb[a];
            }
            dep = pp.deposit != 0;
        }
    }

    // ---- deposit window per axis: the three nodes from start = c0 + min(sh, 0)
    // hold the old and the new shape (sh = cell shift, -1..1); positions in
    // that window: old x0 = o0 + max(-sh, 0), new x1 = o1 + max(sh, 0).
    int start[3], shv[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        shv[a] = dep ? c1[a] - c0[a] : 0;
        start[a] = c0[a] + (shv[a] < 0 ? shv[a] : 0);
    }
    // bounding box of the touched nodes (start .. c0 + 1 + max(sh, 0)):
    // warp minima/maxima first, then one shared atomic per warp
    if (threadIdx.x < 3) {
        bb_lo[threadIdx.x] = 0x7fffffff;
        bb_hi[threadIdx.x] = -0x7fffffff;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int lo_a = __reduce_min_sync(0xffffffffu, dep ? start[a] : 0x7fffffff);
        const int hi_a = __reduce_max_sync(0xffffffffu, dep ? c0[a] + 1 + (shv[a] > 0 ? shv[a] : 0) : -0x7fffffff);
        if ((threadIdx.x & 31) == 0 && lo_a <= hi_a) {
            atomicMin(&bb_lo[a], lo_a);
            atomicMax(&bb_hi[a], hi_a);
        }
    }
    __syncthreads();
    const int w0 = bb_hi[0] - bb_lo[0] + 1, w1 = bb_hi[1] - bb_lo[1] + 1, w2 = bb_hi[2] - bb_lo[2] + 1;
    const bool any = bb_hi[0] >= bb_lo[0];
    const long long box = any ? (long long)w0 * w1 * w2 : 0;
    const bool in_smem = any && 3 * box * (long long)sizeof(T) <= pp.dep_smem;
    const int vol = in_smem ? (int)box : 0;  // nodes in the shared box (32-bit indexing from here)
    if (in_smem) {
        for (int e = threadIdx.x; e < 3 * vol; e += blockDim.x) acc[e] = T(0);
        __syncthreads();
    }
    const int flagv = (int)(step + 1);
    // window width per axis, uniform over the warp: 3 nodes only where some
    // electron of the warp changed cell (mostly along the beam)
    const bool wide_x = __any_sync(0xffffffffu, shv[0] != 0), wide_y = __any_sync(0xffffffffu, shv[1] != 0),
               wide_z = __any_sync(0xffffffffu, shv[2] != 0);
    if (dep) {
        // Esirkepov (linear shapes): old and new shape on the 3-node window
        // (the third node carries no weight when the electron kept its cell)
        T P[3][3], dS[3][3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const T x0 = o0[a] + T(shv[a] < 0 ? -shv[a] : 0);
            const T x1 = o1[a] + T(shv[a] > 0 ? shv[a] : 0);
#pragma unroll
            for (int m = 0; m < 3; m++) {
                const T r0 = T(1) - fabs(x0 - T(m)), r1 = T(1) - fabs(x1 - T(m));
                const T s0 = r0 > T(0) ? r0 : T(0);
                dS[a][m] = (r1 > T(0) ? r1 : T(0)) - s0;
                P[a][m] = s0 + T(0.5) * dS[a][m];
            }
        }
        // shared path: offsets in the block's node box; direct path: offsets
        // of the (wrapped or clamped) window nodes in the grid
        int st[3], l0 = 0;
        long long gofs[3][3];
        if (in_smem) {
            st[0] = 1; st[1] = w0; st[2] = w0 * w1;
            l0 = ((start[2] - bb_lo[2]) * w1 + (start[1] - bb_lo[1])) * w0 + (start[0] - bb_lo[0]);
        } else {
            const long long gs[3] = {1, g.n[0], (long long)g.n[0] * g.n[1]};
            int tl[3][2];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int tsz = a == 0 ? TILE_X : (a == 1 ? TILE_Y : TILE_Z);
#pragma unroll
                for (int m = 0; m < 3; m++) {
                    const int w = wrap_or_clamp<T>(start[a] + m, g.n[a], g.per[a]);
                    gofs[a][m] = w * gs[a];
                    if (m != 1) tl[a][m >> 1] = w / tsz;
                }
            }
            // the window's nodes lie in at most two tiles per axis (its end nodes' tiles)
#pragma unroll
            for (int z = 0; z < 2; z++)
#pragma unroll
                for (int y = 0; y < 2; y++)
#pragma unroll
                    for (int x = 0; x < 2; x++) {
                        if ((z && tl[2][1] == tl[2][0]) || (y && tl[1][1] == tl[1][0]) || (x && tl[0][1] == tl[0][0]))
                            continue;
                        mark_jf_tile(f.jf_flag, f.jf_list, f.jf_count,
                                     ((long long)tl[2][z] * g.nt[1] + tl[1][y]) * g.nt[0] + tl[0][x], flagv);
                    }
        }
        const float fq[3] = {fix_scale(pp.jscale[0]), fix_scale(pp.jscale[1]), fix_scale(pp.jscale[2])};
        if (!wide_y && !wide_z) {
            if (wide_x)
                esirkepov_sites<3, 2, 2>(P, dS, shv, pp.jscale, fq, in_smem, acc, vol, l0, st, f.Jf, gofs);
            else
                esirkepov_sites<2, 2, 2>(P, dS, shv, pp.jscale, fq, in_smem, acc, vol, l0, st, f.Jf, gofs);
        } else {
            esirkepov_sites<3, 3, 3>(P, dS, shv, pp.jscale, fq, in_smem, acc, vol, l0, st, f.Jf, gofs);
        }
    }
    if (in_smem) {
        // Flush: each non-zero entry goes to J_f once.  Lanes of a warp that
        // wrote into the same tile mark it once (the trip count is uniform
        // over the block, so whole warps reach the vote together).
        __syncthreads();
        const int lane = threadIdx.x & 31;
        float iq[3] = {0.f, 0.f, 0.f};  // FP32: the quantum of each component's fixed-point sums
        if constexpr (std::is_same<T, float>::value)
            for (int c = 0; c < 3; c++) iq[c] = (float)(PUSH_BLOCK * fabs(pp.jscale[c])) / FIX_Q;
        for (int e0 = 0; e0 < 3 * vol; e0 += blockDim.x) {
            const int e = e0 + threadIdx.x;
            int tile = -1;
            if (e < 3 * vol) {
                const unsigned c = (unsigned)e / (unsigned)vol;
                T v;
                if constexpr (std::is_same<T, float>::value) {
                    const int iv = reinterpret_cast<const int *>(acc)[e];
                    v = (float)iv * iq[c];
                } else {
                    v = acc[e];
                }
                if (v != T(0)) {
                    const unsigned r = (unsigned)e - c * (unsigned)vol;
                    const unsigned yz = r / (unsigned)w0, z = yz / (unsigned)w1;
                    int idx[3];
                    idx[0] = wrap_or_clamp<T>(bb_lo[0] + (int)(r - yz * (unsigned)w0), g.n[0], g.per[0]);
                    idx[1] = wrap_or_clamp<T>(bb_lo[1] + (int)(yz - z * (unsigned)w1), g.n[1], g.per[1]);
                    idx[2] = wrap_or_clamp<T>(bb_lo[2] + (int)z, g.n[2], g.per[2]);
                    atomicAdd(&f.Jf[c][((long long)idx[2] * g.n[1] + idx[1]) * g.n[0] + idx[0]], v);
                    tile = (int)tile_of(idx, g.nt);
                }
            }
            const unsigned act = __ballot_sync(0xffffffffu, tile >= 0);
            if (tile >= 0) {
                const unsigned grp = __match_any_sync(act, tile);
                if (lane == __ffs(grp) - 1) mark_jf_tile(f.jf_flag, f.jf_list, f.jf_count, tile, flagv);
            }
        }
    }
}

// E^n at x^n for every live electron, taken before the E update
// overwrites E^n (it runs beside the H update, which leaves E alone).
template <typename T>
__global__ void __launch_bounds__(PUSH_BLOCK) k_gather_E(Grid<T> g, Fields<T> f, Particles<T> p) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= p.n || p.status[q]) return;
    int c[3];
    T o[3];
#pragma unroll
    for (int a = 0; a < 3; a++) { c[a] = p.cell[a][q]; o[a] = p.off[a][q]; }
    Stencil<T> st;
    make_stencil(g, c, o, st);
    p.eg[0][q] = interp<1>(f.E[0], g, st);
    p.eg[1][q] = interp<2>(f.E[1], g, st);
    p.eg[2][q] = interp<4>(f.E[2], g, st);
}

template <typename T>
__global__ void k_gather_bold(Grid<T> g, Fields<T> f, Particles<T> p) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= p.n || p.status[q]) return;
    int c[3];
    T o[3];
#pragma unroll
    for (int a = 0; a < 3; a++) { c[a] = p.cell[a][q]; o[a] = p.off[a][q]; }
    Stencil<T> st;
    make_stencil(g, c, o, st);
    T hb[3];
    interp_H(f, g, st, hb);
#pragma unroll
    for (int a = 0; a < 3; a++) p.bold[a][q] = hb[a];
}

// ------------------------------------------------------------ brick sort --
// Lanes of a warp that share a key make one atomic between them: the leader
// adds the group size and each lane gets its own slot from the old value.
// After the first sort most of a warp sits in one brick, so the counters of
// dense bricks see a few atomics instead of one per electron.
__device__ __forceinline__ int warp_grouped_add(int *ctr, int key) {
    const unsigned active = __activemask();
    const unsigned group = __match_any_sync(active, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(group) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&ctr[key], __popc(group));
    base = __shfl_sync(group, base, leader);
    return base + __popc(group & ((1u << lane) - 1));
}

// key = brick of the electron's cell (frozen electrons after all bricks)
template <typename T>
__global__ void k_sort_hist(Particles<T> p, SortBuffers sb) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= p.n) return;
    int key = sb.nbricks;
    if (!p.status[q]) {
        const int bx = p.cell[0][q] / SORT_BRICK, by = p.cell[1][q] / SORT_BRICK, bz = p.cell[2][q] / SORT_BRICK;
        key = (bz * sb.nb[1] + by) * sb.nb[0] + bx;
    }
    sb.key[q] = key;
    warp_grouped_add(sb.count, key);
}

// Exclusive scan of count[0..n) in place, SCAN_TILE entries per block (four
// per thread); each block's total goes to part[].
__global__ void __launch_bounds__(1024) k_scan_tiles(int *count, int n, int *part) {
    __shared__ int s[1024];
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * 4;
    int v[4], sum = 0;
#pragma unroll
    for (int m = 0; m < 4; m++) {
        v[m] = (base + m < n) ? count[base + m] : 0;
        sum += v[m];
    }
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // Hillis-Steele inclusive scan of the thread sums
        const int x = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += x;
        __syncthreads();
    }
    int run = s[threadIdx.x] - sum;  // exclusive prefix of this thread
#pragma unroll
    for (int m = 0; m < 4; m++) {
        if (base + m < n) count[base + m] = run;
        run += v[m];
    }
    if (threadIdx.x == 1023) part[blockIdx.x] = s[1023];
}

// Exclusive scan of the block totals (one block, nparts <= SCAN_TILE).
__global__ void __launch_bounds__(1024) k_scan_parts(int *part, int nparts) {
    __shared__ int s[1024];
    int v[4], sum = 0;
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const int i = threadIdx.x * 4 + m;
        v[m] = i < nparts ? part[i] : 0;
        sum += v[m];
    }
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int x = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += x;
        __syncthreads();
    }
    int run = s[threadIdx.x] - sum;
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const int i = threadIdx.x * 4 + m;
        if (i < nparts) part[i] = run;
        run += v[m];
    }
}

__global__ void __launch_bounds__(1024) k_scan_add(int *count, int n, const int *part) {
    const int add = part[blockIdx.x];
    const int end = min(n, (blockIdx.x + 1) * SCAN_TILE);
    for (int i = blockIdx.x * SCAN_TILE + threadIdx.x; i < end; i += blockDim.x) count[i] += add;
}

// Move each electron to its slot in the scratch arrays (the order inside a
// brick is whatever the atomics give).
template <typename T>
__global__ void k_sort_scatter(Particles<T> p, Particles<T> dst, SortBuffers sb) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= p.n) return;
    const int slot = warp_grouped_add(sb.count, sb.key[q]);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        dst.cell[a][slot] = p.cell[a][q];
        dst.off[a][slot] = p.off[a][q];
        dst.u[a][slot] = p.u[a][q];
        dst.ulo[a][slot] = p.ulo[a][q];
        dst.bold[a][slot] = p.bold[a][q];
    }
    dst.status[slot] = p.status[q];
    dst.id[slot] = p.id[q];
}

template <typename T>
__global__ void k_sort_copyback(Particles<T> p, Particles<T> src) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= p.n) return;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        p.cell[a][q] = src.cell[a][q];
        p.off[a][q] = src.off[a][q];
        p.u[a][q] = src.u[a][q];
        p.ulo[a][q] = src.ulo[a][q];
        p.bold[a][q] = src.bold[a][q];
    }
    p.status[q] = src.status[q];
    p.id[q] = src.id[q];
}

// New electrons [base, base + n) from SI positions and momenta (xyz, u: n x 3
// doubles, copied to the device as given): the (cell, offset) position and
// the compensated momentum in the state precision, input ids, status 0.
// counts[0]: electrons with a non-finite value or outside the allowed
// region (within two cells of a non-periodic face); counts[1]: the others
// whose cell holds a metal (wp > 0).
template <typename T>
__global__ void k_particles_in(const double *xyz, const double *u, long long n, long long base, ParticleIn in,
                               Particles<T> p, const uint8_t *mat, const uint8_t *mat_metal,
                               unsigned long long *counts) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    bool bad = false, metal = false;
    if (q < n) {
        const long long k = base + q;
        int ci[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            double xi = xyz[3 * q + a] / in.d[a];
            const double ua = u[3 * q + a];
            if (!isfinite(xi) || !isfinite(ua)) { bad = true; xi = 0.0; }
            if (in.per[a]) xi -= floor(xi / in.n[a]) * in.n[a];
            const double fl = floor(xi);
            int c = (int)fl;
            const double o = xi - fl;
            if (in.per[a] && c >= in.n[a]) c -= in.n[a];
            if (!in.per[a] && (xi < 2.0 || xi >= in.n[a] - 2.0)) bad = true;
            c = min(max(c, 0), in.n[a] - 1);
            ci[a] = c;
            T ot = (T)o;
            if (ot >= T(1)) ot = nextafter(T(1), T(0));
            const T ut = (T)ua;
            p.cell[a][k] = c;
            p.off[a][k] = ot;
            p.u[a][k] = ut;
            p.ulo[a][k] = (T)(ua - (double)ut);
        }
        p.id[k] = k;
        p.status[k] = 0;
        if (!bad) metal = mat_metal[mat[((long long)ci[2] * in.n[1] + ci[1]) * in.n[0] + ci[0]]] != 0;
    }
    const unsigned bb = __ballot_sync(0xffffffffu, bad), bm = __ballot_sync(0xffffffffu, metal);
    if ((threadIdx.x & 31) == 0) {
        if (bb) atomicAdd(&counts[0], (unsigned long long)__popc(bb));
        if (bm) atomicAdd(&counts[1], (unsigned long long)__popc(bm));
    }
}

template <typename T>
void launch_particles_in(const double *xyz, const double *u, long long n, long long base, const ParticleIn &in,
                         const Particles<T> &p, const uint8_t *mat, const uint8_t *mat_metal,
                         unsigned long long *counts, cudaStream_t s) {
    if (n <= 0) return;
    k_particles_in<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xyz, u, n, base, in, p, mat, mat_metal, counts);
}

template <typename T>
void launch_push_deposit(const Grid<T> &g, const Fields<T> &f, const Particles<T> &p, const PushParams<T> &pp,
                         cudaStream_t s, bool gather_E) {
    if (p.n <= 0) return;
    const unsigned nb = (unsigned)((p.n + PUSH_BLOCK - 1) / PUSH_BLOCK);
    if (gather_E)
        k_push_deposit<T, true><<<nb, PUSH_BLOCK, (size_t)pp.dep_smem, s>>>(g, f, p, pp);
    else
        k_push_deposit<T, false><<<nb, PUSH_BLOCK, (size_t)pp.dep_smem, s>>>(g, f, p, pp);
    launch_count() += 1;
}

template <typename T>
void launch_gather_E(const Grid<T> &g, const Fields<T> &f, const Particles<T> &p, cudaStream_t s) {
    if (p.n <= 0) return;
    k_gather_E<T><<<(unsigned)((p.n + PUSH_BLOCK - 1) / PUSH_BLOCK), PUSH_BLOCK, 0, s>>>(g, f, p);
    launch_count() += 1;
}

template <typename T>
void launch_gather_bold(const Grid<T> &g, const Fields<T> &f, const Particles<T> &p, cudaStream_t s) {
    if (p.n <= 0) return;
    const int blk = 256;
    k_gather_bold<T><<<(unsigned)((p.n + blk - 1) / blk), blk, 0, s>>>(g, f, p);
    launch_count() += 1;
}

template <typename T>
void launch_sort(const Particles<T> &p, const Particles<T> &scratch, const SortBuffers &sb, cudaStream_t s) {
    if (p.n <= 0) return;
    const int blk = 256;
    const unsigned gp = (unsigned)((p.n + blk - 1) / blk);
    const int nbins = sb.nbricks + 1;
    const int ntiles = (nbins + SCAN_TILE - 1) / SCAN_TILE;
    cudaMemsetAsync(sb.count, 0, sizeof(int) * nbins, s);  // a memset node, not a kernel
    k_sort_hist<T><<<gp, blk, 0, s>>>(p, sb);
    launch_count() += 1;
    k_scan_tiles<<<ntiles, 1024, 0, s>>>(sb.count, nbins, sb.part);
    launch_count() += 1;
    k_scan_parts<<<1, 1024, 0, s>>>(sb.part, ntiles);
    launch_count() += 1;
    k_scan_add<<<ntiles, 1024, 0, s>>>(sb.count, nbins, sb.part);
    launch_count() += 1;
    k_sort_scatter<T><<<gp, blk, 0, s>>>(p, scratch, sb);
    launch_count() += 1;
    k_sort_copyback<T><<<gp, blk, 0, s>>>(p, scratch);
    launch_count() += 1;
}

template void launch_particles_in<float>(const double *, const double *, long long, long long, const ParticleIn &,
                                        const Particles<float> &, const uint8_t *, const uint8_t *,
                                        unsigned long long *, cudaStream_t);
template void launch_particles_in<double>(const double *, const double *, long long, long long, const ParticleIn &,
                                         const Particles<double> &, const uint8_t *, const uint8_t *,
                                         unsigned long long *, cudaStream_t);
template void launch_push_deposit<float>(const Grid<float> &, const Fields<float> &, const Particles<float> &,
                                         const PushParams<float> &, cudaStream_t, bool);
template void launch_push_deposit<double>(const Grid<double> &, const Fields<double> &, const Particles<double> &,
                                          const PushParams<double> &, cudaStream_t, bool);
template void launch_gather_E<float>(const Grid<float> &, const Fields<float> &, const Particles<float> &,
                                     cudaStream_t);
template void launch_gather_E<double>(const Grid<double> &, const Fields<double> &, const Particles<double> &,
                                      cudaStream_t);
template void launch_gather_bold<float>(const Grid<float> &, const Fields<float> &, const Particles<float> &,
                                        cudaStream_t);
template void launch_gather_bold<double>(const Grid<double> &, const Fields<double> &, const Particles<double> &,
                                         cudaStream_t);
template void launch_sort<float>(const Particles<float> &, const Particles<float> &, const SortBuffers &, cudaStream_t);
template void launch_sort<double>(const Particles<double> &, const Particles<double> &, const SortBuffers &,
                                  cudaStream_t);

}  // namespace pic
