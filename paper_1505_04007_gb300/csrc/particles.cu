// particles.cu -- electron push and charge-conserving current deposit.
//
// Per live electron, one thread:
//   gather E^n and B^n = mu0 (H^{n-1/2} + H^{n+1/2})/2 at x^n (staggered
//   trilinear; H^{n-1/2}(x^n) is the value the previous push left in bold),
//   relativistic Boris rotation u^{n-1/2} -> u^{n+1/2}, x^{n+1} = x^n + dt u/gamma,
//   the boundary/metal freeze rule, the Esirkepov current of the move
//   (linear node shapes, 4-node window per axis), and finally
//   bold <- H^{n+1/2}(x^{n+1}) for the next step.
// Positions are kept as (integer cell, offset in [0,1)) so FP32 offsets keep
// full relative precision however large the grid.  The momentum is a
// compensated pair (u + ulo): the Boris step is applied as one increment
// du = 2 h E + u' x s (u' = u- + u- x t), which is computed to full relative
// precision, and folded in with an error-free TwoSum, so per-step momentum
// changes that are ~1e-4 of |u| are not truncated by the FP32 mantissa.
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

// Trilinear interpolation of F on a lattice shifted by half a cell along the
// axes flagged in stag (bit a).
template <typename T>
__device__ __forceinline__ T gather(const T *__restrict__ F, const Grid<T> &g, const int c[3], const T o[3],
                                    int stag) {
    int i0[3], i1[3];
    T w[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int b;
        T wa;
        if (stag & (1 << a)) {
            if (o[a] >= T(0.5)) { b = c[a]; wa = o[a] - T(0.5); }
            else { b = c[a] - 1; wa = o[a] + T(0.5); }
        } else {
            b = c[a];
            wa = o[a];
        }
        i0[a] = wrap_or_clamp<T>(b, g.n[a], g.per[a]);
        i1[a] = wrap_or_clamp<T>(b + 1, g.n[a], g.per[a]);
        w[a] = wa;
    }
    const long long nx = g.n[0], nxy = (long long)g.n[0] * g.n[1];
    const long long r00 = i0[2] * nxy + i0[1] * nx, r01 = i0[2] * nxy + i1[1] * nx;
    const long long r10 = i1[2] * nxy + i0[1] * nx, r11 = i1[2] * nxy + i1[1] * nx;
    const T ux = T(1) - w[0], uy = T(1) - w[1], uz = T(1) - w[2];
    const T v00 = ux * F[r00 + i0[0]] + w[0] * F[r00 + i1[0]];
    const T v01 = ux * F[r01 + i0[0]] + w[0] * F[r01 + i1[0]];
    const T v10 = ux * F[r10 + i0[0]] + w[0] * F[r10 + i1[0]];
    const T v11 = ux * F[r11 + i0[0]] + w[0] * F[r11 + i1[0]];
    return uz * (uy * v00 + w[1] * v01) + w[2] * (uy * v10 + w[1] * v11);
}

// stagger bits: Ex x, Ey y, Ez z; Hx y|z, Hy x|z, Hz x|y
__device__ __constant__ int STAG_E[3] = {1, 2, 4};
__device__ __constant__ int STAG_H[3] = {6, 5, 3};

template <typename T>
__device__ __forceinline__ void shape4(T x, T S[4]) {
#pragma unroll
    for (int m = 0; m < 4; m++) {
        T r = T(1) - fabs(x - T(m));
        S[m] = r > T(0) ? r : T(0);
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_push_deposit(Grid<T> g, Fields<T> f, Particles<T> p, PushParams<T> pp) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= p.n || p.status[q]) return;
    const long long step = *f.step;

    int c0[3];
    T o0[3], u[3], ul[3], E[3], B[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        c0[a] = p.cell[a][q]; o0[a] = p.off[a][q]; u[a] = p.u[a][q]; ul[a] = p.ulo[a][q];
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        E[a] = gather(f.E[a], g, c0, o0, STAG_E[a]);
        const T hnew = gather(f.H[a], g, c0, o0, STAG_H[a]);
        B[a] = pp.mu0 * T(0.5) * (p.bold[a][q] + hnew);
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
    if (!isfinite(gn)) { atomicOr(pp.err, DEVERR_NONFINITE); p.status[q] = 1; return; }
    const T ig = T(1) / gn;

    // move in (cell, offset) form; raw cell before periodic wrap for the deposit
    int c1[3], c1w[3];
    T o1[3];
    bool frozen = false;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        T x = o0[a] + (un[a] + unl[a]) * pp.dtd[a] * ig;
        T fl = floor(x);
        int sh = (int)fl;
        x -= fl;
        if (x >= T(1)) { x -= T(1); sh += 1; }
        if (sh < -1 || sh > 1) { atomicOr(pp.err, DEVERR_JUMP); frozen = true; }
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
    if (frozen) { p.status[q] = 1; return; }

    if (pp.deposit) {
        T S0[3][4], dS[3][4];
        int base[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            base[a] = c0[a] - 1;
            T S1[4];
            shape4(T(1) + o0[a], S0[a]);
            shape4(T(c1[a] - c0[a] + 1) + o1[a], S1);
#pragma unroll
            for (int m = 0; m < 4; m++) dS[a][m] = S1[m] - S0[a][m];
        }
        const int flagv = (int)(step + 1);
        const T third = T(1) / T(3);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
            T *J = f.Jf[c];
            for (int m2 = 0; m2 < 4; m2++) {
                for (int m1 = 0; m1 < 4; m1++) {
                    const T tr = S0[a1][m1] * S0[a2][m2] + T(0.5) * dS[a1][m1] * S0[a2][m2] +
                                 T(0.5) * S0[a1][m1] * dS[a2][m2] + third * dS[a1][m1] * dS[a2][m2];
                    if (tr == T(0)) continue;
                    int idx[3];
                    idx[a1] = wrap_or_clamp<T>(base[a1] + m1, g.n[a1], g.per[a1]);
                    idx[a2] = wrap_or_clamp<T>(base[a2] + m2, g.n[a2], g.per[a2]);
                    T acc = T(0);
#pragma unroll
                    for (int m0 = 0; m0 < 3; m0++) {
                        acc += dS[c][m0] * tr;
                        if (acc == T(0)) continue;
                        idx[c] = wrap_or_clamp<T>(base[c] + m0, g.n[c], g.per[c]);
                        const long long e = ((long long)idx[2] * g.n[1] + idx[1]) * g.n[0] + idx[0];
                        atomicAdd(&J[e], pp.jscale[c] * acc);
                        const long long tl = ((long long)(idx[2] / TILE_Z) * g.nt[1] + idx[1] / TILE_Y) * g.nt[0] +
                                             idx[0] / TILE_X;
                        f.jf_flag[tl] = flagv;
                    }
                }
            }
        }
    }

#pragma unroll
    for (int a = 0; a < 3; a++) {
        p.cell[a][q] = c1w[a];
        p.off[a][q] = o1[a];
        p.u[a][q] = un[a];
        p.ulo[a][q] = unl[a];
    }
#pragma unroll
    for (int a = 0; a < 3; a++) p.bold[a][q] = gather(f.H[a], g, c1w, o1, STAG_H[a]);
}

template <typename T>
__global__ void k_gather_bold(Grid<T> g, Fields<T> f, Particles<T> p) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= p.n || p.status[q]) return;
    int c[3];
    T o[3];
#pragma unroll
    for (int a = 0; a < 3; a++) { c[a] = p.cell[a][q]; o[a] = p.off[a][q]; }
#pragma unroll
    for (int a = 0; a < 3; a++) p.bold[a][q] = gather(f.H[a], g, c, o, STAG_H[a]);
}

template <typename T>
void launch_push_deposit(const Grid<T> &g, const Fields<T> &f, const Particles<T> &p, const PushParams<T> &pp,
                         cudaStream_t s) {
    if (p.n <= 0) return;
    const int blk = 128;
    k_push_deposit<T><<<(unsigned)((p.n + blk - 1) / blk), blk, 0, s>>>(g, f, p, pp);
}

template <typename T>
void launch_gather_bold(const Grid<T> &g, const Fields<T> &f, const Particles<T> &p, cudaStream_t s) {
    if (p.n <= 0) return;
    const int blk = 256;
    k_gather_bold<T><<<(unsigned)((p.n + blk - 1) / blk), blk, 0, s>>>(g, f, p);
}

template void launch_push_deposit<float>(const Grid<float> &, const Fields<float> &, const Particles<float> &,
                                         const PushParams<float> &, cudaStream_t);
template void launch_push_deposit<double>(const Grid<double> &, const Fields<double> &, const Particles<double> &,
                                          const PushParams<double> &, cudaStream_t);
template void launch_gather_bold<float>(const Grid<float> &, const Fields<float> &, const Particles<float> &,
                                        cudaStream_t);
template void launch_gather_bold<double>(const Grid<double> &, const Fields<double> &, const Particles<double> &,
                                         cudaStream_t);

}  // namespace pic
