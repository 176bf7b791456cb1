// adjoint.cu -- gradient of a probe's plasmon spectral energy with respect
// to the film's Drude mask, wp and gamma (include/pic_adjoint.h).
//
// Forward: the field part of the PIC step (H with CPML; Eq. 6 then Eq. 8
// with CPML), the electrons replaced by a rigid Gaussian bunch current, a
// per-edge Drude factor bJ built from a per-cell mask.  Backward: the exact
// transpose of that step, run from the last step to the first.  Each
// forward update is a sum of terms "target += c * source"; its transpose
// adds c * adjoint(target) to adjoint(source).  The transposed H and E
// updates scatter into the neighbours' adjoint values with atomics (several
// cells read the same neighbour in the forward step), the CPML psi and the
// Drude current J are per-edge states whose adjoints stay in place.
// Every E^n and J^n on the design edges is stored during the forward run
// (nothing is recomputed); gradients of bJ and kJ accumulate in FP64 per
// design edge and are reduced to the mask, wp and gamma on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "../../include/pic.h"
#include "../../include/pic_adjoint.h"
#include "pic_internal.cuh"

namespace pic {
namespace {

template <typename T>
struct AGrid {
    int n[3];
    int L;       // CPML cells on every face
    T r[3];      // 1/dx per axis
    T cH, cE;    // dt/mu0, dt/eps0
    T kJm1;      // kJ - 1 (uniform gamma)
    int ks0, ks1;  // cell planes [ks0, ks1) hold every design edge
};

template <typename T>
struct AState {
    T *E[3], *H[3], *J[3];
    T *psiH[3][2], *psiE[3][2];  // same compact slab layout as the main path
    T *lE[3], *lH[3], *lJ[3];    // adjoints
    T *lpsiH[3][2], *lpsiE[3][2];
    const T *bE[3], *aE[3], *ikE[3], *bH[3], *aH[3], *ikH[3];  // b-1, a, 1/kappa
    const int *slot[3];          // per edge: design-edge slot, or -1
    const long long *eidx;       // per slot: linear edge index
    long long soff[4];           // slots of component c are [soff[c], soff[c+1])
    const T *beta;               // per slot: bJ
    T *stE, *stJ;                // per step and slot: E^n, J^n
    double *gb, *gk;             // per slot: dL/dbJ, dL/dkJ contributions
    long long *n;                // device step counter (forward: next step; backward: steps left)
    long long seg;               // steps n with rows n % seg in the storage (all steps, or one segment)
};

// The rigid bunch's current on the Ex edges at t = (n + 1/2) dt,
//   J_x(i+1/2, j, k) = q v (2 pi s^2)^{-3/2} exp(-r^2 / (2 s^2)),
// on every edge of the grid (it is zero only where the Gaussian underflows).
// The Gaussian factorises: J_x = gx[n][i] * gyz[k][j] with
//   gx[n][i] = exp(-((i + 1/2) dx - x0 - v t)^2 / (2 s^2))
//   gyz[k][j] = q v (2 pi s^2)^{-3/2} exp(-((j dx - y0)^2 + (k dx - z0)^2) / (2 s^2)),
// both evaluated in FP64 on the host at create (every step of the run), so an
// edge costs one multiply instead of an FP64 exponential.
struct Bunch {
    const double *gx64, *gyz64;  // FP64 state
    const float *gx32, *gyz32;   // FP32 state: the FP64 factors rounded to float
    int nx, ny;
    long long nsteps;
};

struct Probe {
    long long idx[8];
    double w[8];
    int lo[3], hi[3];  // cell index range of the eight corners per axis
    int comp;
    double omega, dt;
};

// F += E_c(x_p, t) exp(+i omega t) dt at t = (n+1) dt (the probe DFT at one
// frequency, from E^{n+1})
template <typename T>
__device__ __forceinline__ void probe_term(const AState<T> &f, const Probe &p, double *F, long long n) {
    const double t = (n + 1) * p.dt;
    double v = 0.0;
    for (int q = 0; q < 8; q++) v += p.w[q] * (double)f.E[p.comp][p.idx[q]];
    double sn, cs;
    sincos(p.omega * t, &sn, &cs);
    F[0] += v * cs * p.dt;
    F[1] += v * sn * p.dt;
}

// Start of forward step m (one thread): the probe term of step m-1 and the
// counter from m-1 to m.
template <typename T>
__device__ __forceinline__ void fwd_step_start(const AState<T> &f, const Probe &pr, double *F) {
    const long long m1 = *f.n;
    if (m1 >= 0) probe_term(f, pr, F, m1);
    *f.n = m1 + 1;
}

__device__ __forceinline__ int aslab(int L, int n, int x) {
    if (x < L) return x;
    if (x >= n - L) return x - (n - 2 * L);
    return -1;
}
__device__ __forceinline__ long long apsi(const int n[3], int L, int a, int s, int i, int j, int k) {
    const long long L2 = 2 * L;
    if (a == 0) return ((long long)k * n[1] + j) * L2 + s;
    if (a == 1) return ((long long)k * L2 + s) * n[0] + i;
    return ((long long)s * n[1] + j) * n[0] + i;
}

// ------------------------------------------------------------ forward --
// Step m starts here.  Its first thread also takes the probe term of step
// m-1 (E is E^m until the E update that follows) and advances the step
// counter from m-1 to m (it starts at -1).
template <typename T>
__global__ void __launch_bounds__(256) k_fwd_H(AGrid<T> g, AState<T> f, Probe pr, double *F, Bunch bu, double dt) {
    pdl_wait();
    pdl_release();
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0) fwd_step_start(f, pr, F);
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (i >= nx || j >= ny) return;
    const long long sy = nx, sz = (long long)nx * ny, e = k * sz + j * sy + i;
    const T ex = f.E[0][e], ey = f.E[1][e], ez = f.E[2][e];
    const T dEz_dy = ((j + 1 < ny ? f.E[2][e + sy] : T(0)) - ez) * g.r[1];
    const T dEy_dz = ((k + 1 < nz ? f.E[1][e + sz] : T(0)) - ey) * g.r[2];
    const T dEx_dz = ((k + 1 < nz ? f.E[0][e + sz] : T(0)) - ex) * g.r[2];
    const T dEz_dx = ((i + 1 < nx ? f.E[2][e + 1] : T(0)) - ez) * g.r[0];
    const T dEy_dx = ((i + 1 < nx ? f.E[1][e + 1] : T(0)) - ey) * g.r[0];
    const T dEx_dy = ((j + 1 < ny ? f.E[0][e + sy] : T(0)) - ex) * g.r[1];
    T kx = 1, ky = 1, kz = 1, pxy = 0, pxz = 0, pyz = 0, pyx = 0, pzx = 0, pzy = 0;
    const int s0 = aslab(g.L, nx, i), s1 = aslab(g.L, ny, j), s2 = aslab(g.L, nz, k);
    if (s0 >= 0) {
        const T b = f.bH[0][i], a = f.aH[0][i];
        kx = f.ikH[0][i];
        const long long q = apsi(g.n, g.L, 0, s0, i, j, k);
        pxy = f.psiH[0][0][q] + (b * f.psiH[0][0][q] + a * dEz_dx); f.psiH[0][0][q] = pxy;
        pxz = f.psiH[0][1][q] + (b * f.psiH[0][1][q] + a * dEy_dx); f.psiH[0][1][q] = pxz;
    }
    if (s1 >= 0) {
        const T b = f.bH[1][j], a = f.aH[1][j];
        ky = f.ikH[1][j];
        const long long q = apsi(g.n, g.L, 1, s1, i, j, k);
        pyz = f.psiH[1][0][q] + (b * f.psiH[1][0][q] + a * dEx_dy); f.psiH[1][0][q] = pyz;
        pyx = f.psiH[1][1][q] + (b * f.psiH[1][1][q] + a * dEz_dy); f.psiH[1][1][q] = pyx;
    }
    if (s2 >= 0) {
        const T b = f.bH[2][k], a = f.aH[2][k];
        kz = f.ikH[2][k];
        const long long q = apsi(g.n, g.L, 2, s2, i, j, k);
        pzx = f.psiH[2][0][q] + (b * f.psiH[2][0][q] + a * dEy_dz); f.psiH[2][0][q] = pzx;
        pzy = f.psiH[2][1][q] + (b * f.psiH[2][1][q] + a * dEx_dz); f.psiH[2][1][q] = pzy;
    }
    f.H[0][e] -= g.cH * (ky * dEz_dy + pyx - kz * dEy_dz - pzx);
    f.H[1][e] -= g.cH * (kz * dEx_dz + pzy - kx * dEz_dx - pxy);
    f.H[2][e] -= g.cH * (kx * dEy_dx + pxz - ky * dEx_dy - pyz);
}

// the rigid bunch current J_x at the Ex edge (i+1/2, j, k) in step n
// (t = (n + 1/2) dt), in the state precision
template <typename T>
__device__ __forceinline__ T bunch_jx(const Bunch &b, int i, int j, int k, long long n);
template <>
__device__ __forceinline__ double bunch_jx<double>(const Bunch &b, int i, int j, int k, long long n) {
    if (n < 0 || n >= b.nsteps) return 0.0;
    return b.gx64[n * b.nx + i] * b.gyz64[(long long)k * b.ny + j];
}
template <>
__device__ __forceinline__ float bunch_jx<float>(const Bunch &b, int i, int j, int k, long long n) {
    if (n < 0 || n >= b.nsteps) return 0.f;
    return b.gx32[n * b.nx + i] * b.gyz32[(long long)k * b.ny + j];
}

template <typename T>
__device__ __forceinline__ int design_slot(const AGrid<T> &g, const AState<T> &f, int c, long long e, int k) {
    return (k >= g.ks0 && k < g.ks1) ? f.slot[c][e] : -1;
}

// Eq. 6 (design edges) then Eq. 8 for component c of edge e at plane k;
// E^n and J^n of a design edge go to storage row n % seg (nr) on the way
template <typename T>
__device__ __forceinline__ void fwd_ampere(const AGrid<T> &g, const AState<T> &f, int c, long long e, int k,
                                           long long nr, T curl, T js) {
    T E = f.E[c][e], jp = T(0);
    const int sl = design_slot(g, f, c, e, k);
    if (sl >= 0) {
        const T j0 = f.J[c][e];
        const long long row = nr * f.soff[3] + sl;
        f.stE[row] = E;
        f.stJ[row] = j0;
        jp = j0 + (g.kJm1 * j0 + f.beta[sl] * E);
        f.J[c][e] = jp;
    }
    f.E[c][e] = E + g.cE * (curl - jp - js);
}

template <typename T>
__global__ void __launch_bounds__(256) k_fwd_E(AGrid<T> g, AState<T> f, Bunch bu, double dt) {
    pdl_wait();
    pdl_release();
    const long long n = *f.n, nr = n % f.seg;
    (void)dt;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (i >= nx || j >= ny) return;
    const long long sy = nx, sz = (long long)nx * ny, e = k * sz + j * sy + i;
    const bool fx = i == 0, fy = j == 0, fz = k == 0;  // held tangential E on the low faces
    const long long oim = i > 0 ? 1 : 0, ojm = j > 0 ? sy : 0, okm = k > 0 ? sz : 0;
    const T hx = f.H[0][e], hy = f.H[1][e], hz = f.H[2][e];
    const int s0 = aslab(g.L, nx, i), s1 = aslab(g.L, ny, j), s2 = aslab(g.L, nz, k);
    if (!(fy || fz)) {
        const T dHz_dy = (hz - f.H[2][e - ojm]) * g.r[1], dHy_dz = (hy - f.H[1][e - okm]) * g.r[2];
        T ky = 1, kz = 1, py = 0, pz = 0;
        if (s1 >= 0) {
            ky = f.ikE[1][j];
            const long long q = apsi(g.n, g.L, 1, s1, i, j, k);
            py = f.psiE[1][1][q] + (f.bE[1][j] * f.psiE[1][1][q] + f.aE[1][j] * dHz_dy); f.psiE[1][1][q] = py;
        }
        if (s2 >= 0) {
            kz = f.ikE[2][k];
            const long long q = apsi(g.n, g.L, 2, s2, i, j, k);
            pz = f.psiE[2][0][q] + (f.bE[2][k] * f.psiE[2][0][q] + f.aE[2][k] * dHy_dz); f.psiE[2][0][q] = pz;
        }
        fwd_ampere(g, f, 0, e, k, nr, ky * dHz_dy + py - kz * dHy_dz - pz, bunch_jx<T>(bu, i, j, k, n));
    }
    if (!(fx || fz)) {
        const T dHx_dz = (hx - f.H[0][e - okm]) * g.r[2], dHz_dx = (hz - f.H[2][e - oim]) * g.r[0];
        T kz = 1, kx = 1, pz = 0, px = 0;
        if (s2 >= 0) {
            kz = f.ikE[2][k];
            const long long q = apsi(g.n, g.L, 2, s2, i, j, k);
            pz = f.psiE[2][1][q] + (f.bE[2][k] * f.psiE[2][1][q] + f.aE[2][k] * dHx_dz); f.psiE[2][1][q] = pz;
        }
        if (s0 >= 0) {
            kx = f.ikE[0][i];
            const long long q = apsi(g.n, g.L, 0, s0, i, j, k);
            px = f.psiE[0][0][q] + (f.bE[0][i] * f.psiE[0][0][q] + f.aE[0][i] * dHz_dx); f.psiE[0][0][q] = px;
        }
        fwd_ampere(g, f, 1, e, k, nr, kz * dHx_dz + pz - kx * dHz_dx - px, T(0));
    }
    if (!(fx || fy)) {
        const T dHy_dx = (hy - f.H[1][e - oim]) * g.r[0], dHx_dy = (hx - f.H[0][e - ojm]) * g.r[1];
        T kx = 1, ky = 1, px = 0, py = 0;
        if (s0 >= 0) {
            kx = f.ikE[0][i];
            const long long q = apsi(g.n, g.L, 0, s0, i, j, k);
            px = f.psiE[0][1][q] + (f.bE[0][i] * f.psiE[0][1][q] + f.aE[0][i] * dHy_dx); f.psiE[0][1][q] = px;
        }
        if (s1 >= 0) {
            ky = f.ikE[1][j];
            const long long q = apsi(g.n, g.L, 1, s1, i, j, k);
            py = f.psiE[1][0][q] + (f.bE[1][j] * f.psiE[1][0][q] + f.aE[1][j] * dHx_dy); f.psiE[1][0][q] = py;
        }
        fwd_ampere(g, f, 2, e, k, nr, kx * dHy_dx + px - ky * dHx_dy - py, T(0));
    }
}

// the step counter set on the device (kept in stream order with the steps)
__global__ void k_set_counter(long long *n, long long v) {
    if (threadIdx.x == 0) *n = v;
}

// the probe term of the last step, after the last E update
template <typename T>
__global__ void k_probe(AState<T> f, Probe p, double *F) {
    if (threadIdx.x != 0) return;
    const long long n = *f.n;
    probe_term(f, p, F, n);
    *f.n = n + 1;
}

// ----------------------------------------------------------- backward --
// Adjoint of the probe term of step n at t = (n+1) dt, added by the thread
// that owns edge e of the probed component before it reads lambda_E:
// dL/dE = 2 Re(conj(F) e^{i omega t}) dt w
template <typename T>
__device__ __forceinline__ void probe_source(const AState<T> &f, const Probe &p, const double *F, long long n, int i,
                                             int j, int k, long long e) {
    if (i < p.lo[0] || i > p.hi[0] || j < p.lo[1] || j > p.hi[1] || k < p.lo[2] || k > p.hi[2]) return;
    const double t = (n + 1) * p.dt;
    double sn, cs;
    sincos(p.omega * t, &sn, &cs);
    const double s = 2.0 * p.dt * (F[0] * cs + F[1] * sn);
    for (int q = 0; q < 8; q++)
        if (p.idx[q] == e) f.lE[p.comp][e] += (T)(s * p.w[q]);
}

// Transpose of the Eq. 6 + Eq. 8 update of component c at edge e (updated
// edges only).  Returns nothing; updates the adjoints of E, J (in place) and
// accumulates the bJ / kJ gradients with the stored E^n, J^n.
template <typename T>
__device__ __forceinline__ void adj_ampere(const AGrid<T> &g, const AState<T> &f, int c, long long e, int k, T lE,
                                           long long nr) {
    const int sl = design_slot(g, f, c, e, k);
    if (sl < 0) return;  // lambda_E passes through unchanged
    const long long ne = f.soff[3];
    const T LJ = f.lJ[c][e] - g.cE * lE;  // adjoint of J^{n+1}
    f.gb[sl] += (double)LJ * (double)f.stE[nr * ne + sl];
    f.gk[sl] += (double)LJ * (double)f.stJ[nr * ne + sl];
    f.lJ[c][e] = (T(1) + g.kJm1) * LJ;
    f.lE[c][e] = lE + f.beta[sl] * LJ;
}

// Backward step n = (steps left) - 1; k_adj_H then stores n as the counter.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_E(AGrid<T> g, AState<T> f, Probe pr, const double *F) {
    pdl_wait();
    pdl_release();
    const long long n = *f.n - 1, nr = n % f.seg;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (i >= nx || j >= ny) return;
    const long long sy = nx, sz = (long long)nx * ny, e = k * sz + j * sy + i;
    probe_source(f, pr, F, n, i, j, k, e);
    const bool fx = i == 0, fy = j == 0, fz = k == 0;
    const int s0 = aslab(g.L, nx, i), s1 = aslab(g.L, ny, j), s2 = aslab(g.L, nz, k);
    const T cE = g.cE;
    // scatter A * d(H_c)/d... for a backward difference (H[e] - H[e - off]) * r
    auto scat = [&](T *lH, long long off, bool has, T r, T A) {
        atomicAdd(&lH[e], r * A);
        if (has) atomicAdd(&lH[e - off], -r * A);
    };
    if (!(fy || fz)) {  // Ex: curl = ky dHz/dy + py - kz dHy/dz - pz
        const T lE = f.lE[0][e];
        T Ay = cE * lE, Az = -cE * lE;
        if (s1 >= 0) {
            const long long q = apsi(g.n, g.L, 1, s1, i, j, k);
            const T ap = f.lpsiE[1][1][q] + cE * lE;
            Ay = cE * f.ikE[1][j] * lE + f.aE[1][j] * ap;
            f.lpsiE[1][1][q] = (T(1) + f.bE[1][j]) * ap;
        }
        if (s2 >= 0) {
            const long long q = apsi(g.n, g.L, 2, s2, i, j, k);
            const T ap = f.lpsiE[2][0][q] - cE * lE;
            Az = -cE * f.ikE[2][k] * lE + f.aE[2][k] * ap;
            f.lpsiE[2][0][q] = (T(1) + f.bE[2][k]) * ap;
        }
        scat(f.lH[2], sy, j > 0, g.r[1], Ay);
        scat(f.lH[1], sz, k > 0, g.r[2], Az);
        adj_ampere(g, f, 0, e, k, lE, nr);
    }
    if (!(fx || fz)) {  // Ey: curl = kz dHx/dz + pz - kx dHz/dx - px
        const T lE = f.lE[1][e];
        T Az = cE * lE, Ax = -cE * lE;
        if (s2 >= 0) {
            const long long q = apsi(g.n, g.L, 2, s2, i, j, k);
            const T ap = f.lpsiE[2][1][q] + cE * lE;
            Az = cE * f.ikE[2][k] * lE + f.aE[2][k] * ap;
            f.lpsiE[2][1][q] = (T(1) + f.bE[2][k]) * ap;
        }
        if (s0 >= 0) {
            const long long q = apsi(g.n, g.L, 0, s0, i, j, k);
            const T ap = f.lpsiE[0][0][q] - cE * lE;
            Ax = -cE * f.ikE[0][i] * lE + f.aE[0][i] * ap;
            f.lpsiE[0][0][q] = (T(1) + f.bE[0][i]) * ap;
        }
        scat(f.lH[0], sz, k > 0, g.r[2], Az);
        scat(f.lH[2], 1, i > 0, g.r[0], Ax);
        adj_ampere(g, f, 1, e, k, lE, nr);
    }
    if (!(fx || fy)) {  // Ez: curl = kx dHy/dx + px - ky dHx/dy - py
        const T lE = f.lE[2][e];
        T Ax = cE * lE, Ay = -cE * lE;
        if (s0 >= 0) {
            const long long q = apsi(g.n, g.L, 0, s0, i, j, k);
            const T ap = f.lpsiE[0][1][q] + cE * lE;
            Ax = cE * f.ikE[0][i] * lE + f.aE[0][i] * ap;
            f.lpsiE[0][1][q] = (T(1) + f.bE[0][i]) * ap;
        }
        if (s1 >= 0) {
            const long long q = apsi(g.n, g.L, 1, s1, i, j, k);
            const T ap = f.lpsiE[1][0][q] - cE * lE;
            Ay = -cE * f.ikE[1][j] * lE + f.aE[1][j] * ap;
            f.lpsiE[1][0][q] = (T(1) + f.bE[1][j]) * ap;
        }
        scat(f.lH[1], 1, i > 0, g.r[0], Ax);
        scat(f.lH[0], sy, j > 0, g.r[1], Ay);
        adj_ampere(g, f, 2, e, k, lE, nr);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_H(AGrid<T> g, AState<T> f) {
    pdl_wait();
    pdl_release();
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0) *f.n -= 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (i >= nx || j >= ny) return;
    const long long sy = nx, sz = (long long)nx * ny, e = k * sz + j * sy + i;
    const T lx = f.lH[0][e], ly = f.lH[1][e], lz = f.lH[2][e], cH = g.cH;
    // adjoints of the six differences (forward differences of E)
    T Azy = -cH * lx, Ayz = cH * lx, Axz = -cH * ly, Azx = cH * ly, Ayx = -cH * lz, Axy = cH * lz;
    const int s0 = aslab(g.L, nx, i), s1 = aslab(g.L, ny, j), s2 = aslab(g.L, nz, k);
    if (s0 >= 0) {
        const T a = f.aH[0][i], k0 = f.ikH[0][i], b1 = T(1) + f.bH[0][i];
        const long long q = apsi(g.n, g.L, 0, s0, i, j, k);
        const T pxy = f.lpsiH[0][0][q] + cH * ly, pxz = f.lpsiH[0][1][q] - cH * lz;
        Azx = cH * k0 * ly + a * pxy;
        Ayx = -cH * k0 * lz + a * pxz;
        f.lpsiH[0][0][q] = b1 * pxy;
        f.lpsiH[0][1][q] = b1 * pxz;
    }
    if (s1 >= 0) {
        const T a = f.aH[1][j], k1 = f.ikH[1][j], b1 = T(1) + f.bH[1][j];
        const long long q = apsi(g.n, g.L, 1, s1, i, j, k);
        const T pyz = f.lpsiH[1][0][q] + cH * lz, pyx = f.lpsiH[1][1][q] - cH * lx;
        Axy = cH * k1 * lz + a * pyz;
        Azy = -cH * k1 * lx + a * pyx;
        f.lpsiH[1][0][q] = b1 * pyz;
        f.lpsiH[1][1][q] = b1 * pyx;
    }
    if (s2 >= 0) {
        const T a = f.aH[2][k], k2 = f.ikH[2][k], b1 = T(1) + f.bH[2][k];
        const long long q = apsi(g.n, g.L, 2, s2, i, j, k);
        const T pzx = f.lpsiH[2][0][q] + cH * lx, pzy = f.lpsiH[2][1][q] - cH * ly;
        Ayz = cH * k2 * lx + a * pzx;
        Axz = -cH * k2 * ly + a * pzy;
        f.lpsiH[2][0][q] = b1 * pzx;
        f.lpsiH[2][1][q] = b1 * pzy;
    }
    // d = (E[e + off] - E[e]) * r, E[e + off] = 0 beyond the high face
    auto scat = [&](T *lE, long long off, bool has, T r, T A) {
        if (has) atomicAdd(&lE[e + off], r * A);
        atomicAdd(&lE[e], -r * A);
    };
    scat(f.lE[2], sy, j + 1 < ny, g.r[1], Azy);
    scat(f.lE[1], sz, k + 1 < nz, g.r[2], Ayz);
    scat(f.lE[0], sz, k + 1 < nz, g.r[2], Axz);
    scat(f.lE[2], 1, i + 1 < nx, g.r[0], Azx);
    scat(f.lE[1], 1, i + 1 < nx, g.r[0], Ayx);
    scat(f.lE[0], sy, j + 1 < ny, g.r[1], Axy);
}

// ------------------------------------------- FP32, four cells per thread --
// The forward H and E kernels and the transposed H update for FP32 state with
// four consecutive x cells per thread (nx and the CPML width multiples of 4,
// so a group lies wholly inside or outside the x slabs): every centre, row
// and plane access is one 16-byte load or store, and the transposed H update
// adds into a neighbouring group with one 16-byte atomic instead of four (the
// contributions a group makes to its own cells are summed first).  Per cell
// the arithmetic is that of the kernels above; only the order of the atomic
// sums differs.  The transposed E update keeps the one-cell kernel: its
// four-cell form measured slower (35.7 against 31.1 us per launch at
// 192x96x96).
struct V4 {
    float v[4];
};
__device__ __forceinline__ V4 ld4(const float *p) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    return V4{{q.x, q.y, q.z, q.w}};
}
__device__ __forceinline__ void st4(float *p, const V4 &a) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
__device__ __forceinline__ void add4(float *p, const V4 &a) {
    atomicAdd(reinterpret_cast<float4 *>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
}
__device__ __forceinline__ V4 zero4() { return V4{{0.f, 0.f, 0.f, 0.f}}; }

__device__ __forceinline__ bool group_of(const AGrid<float> &g, int &i0, int &j, int &k) {
    i0 = 4 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    j = blockIdx.y * blockDim.y + threadIdx.y;
    k = blockIdx.z;
    return i0 < g.n[0] && j < g.n[1];
}

__global__ void __launch_bounds__(256) k_fwd_H4(AGrid<float> g, AState<float> f, Probe pr, double *F, Bunch bu,
                                                 double dt) {
    pdl_wait();
    pdl_release();
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0) fwd_step_start(f, pr, F);
    int i0, j, k;
    if (!group_of(g, i0, j, k)) return;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long sy = nx, sz = (long long)nx * ny, e = k * sz + j * sy + i0;
    const V4 ex = ld4(f.E[0] + e), ey = ld4(f.E[1] + e), ez = ld4(f.E[2] + e);
    const V4 ez_jp = j + 1 < ny ? ld4(f.E[2] + e + sy) : zero4(), ex_jp = j + 1 < ny ? ld4(f.E[0] + e + sy) : zero4();
    const V4 ey_kp = k + 1 < nz ? ld4(f.E[1] + e + sz) : zero4(), ex_kp = k + 1 < nz ? ld4(f.E[0] + e + sz) : zero4();
    const float ez_ip = i0 + 4 < nx ? f.E[2][e + 4] : 0.f, ey_ip = i0 + 4 < nx ? f.E[1][e + 4] : 0.f;
    V4 hx = ld4(f.H[0] + e), hy = ld4(f.H[1] + e), hz = ld4(f.H[2] + e);
    const float rx = g.r[0], ry = g.r[1], rz = g.r[2];
    float dEz_dy[4], dEy_dz[4], dEx_dz[4], dEz_dx[4], dEy_dx[4], dEx_dy[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        dEz_dy[m] = (ez_jp.v[m] - ez.v[m]) * ry;
        dEy_dz[m] = (ey_kp.v[m] - ey.v[m]) * rz;
        dEx_dz[m] = (ex_kp.v[m] - ex.v[m]) * rz;
        dEz_dx[m] = ((m < 3 ? ez.v[m + 1] : ez_ip) - ez.v[m]) * rx;
        dEy_dx[m] = ((m < 3 ? ey.v[m + 1] : ey_ip) - ey.v[m]) * rx;
        dEx_dy[m] = (ex_jp.v[m] - ex.v[m]) * ry;
    }
    float kx[4] = {1.f, 1.f, 1.f, 1.f}, ky = 1.f, kz = 1.f;
    V4 pxy = zero4(), pxz = zero4(), pyz = zero4(), pyx = zero4(), pzx = zero4(), pzy = zero4();
    const int s0 = aslab(g.L, nx, i0), s1 = aslab(g.L, ny, j), s2 = aslab(g.L, nz, k);
    if (s0 >= 0) {
        const long long q = apsi(g.n, g.L, 0, s0, i0, j, k);
        const V4 o0 = ld4(f.psiH[0][0] + q), o1 = ld4(f.psiH[0][1] + q);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const float b = f.bH[0][i0 + m], a = f.aH[0][i0 + m];
            kx[m] = f.ikH[0][i0 + m];
            pxy.v[m] = o0.v[m] + (b * o0.v[m] + a * dEz_dx[m]);
            pxz.v[m] = o1.v[m] + (b * o1.v[m] + a * dEy_dx[m]);
        }
        st4(f.psiH[0][0] + q, pxy);
        st4(f.psiH[0][1] + q, pxz);
    }
    if (s1 >= 0) {
        const float b = f.bH[1][j], a = f.aH[1][j];
        ky = f.ikH[1][j];
        const long long q = apsi(g.n, g.L, 1, s1, i0, j, k);
        const V4 o0 = ld4(f.psiH[1][0] + q), o1 = ld4(f.psiH[1][1] + q);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            pyz.v[m] = o0.v[m] + (b * o0.v[m] + a * dEx_dy[m]);
            pyx.v[m] = o1.v[m] + (b * o1.v[m] + a * dEz_dy[m]);
        }
        st4(f.psiH[1][0] + q, pyz);
        st4(f.psiH[1][1] + q, pyx);
    }
    if (s2 >= 0) {
        const float b = f.bH[2][k], a = f.aH[2][k];
        kz = f.ikH[2][k];
        const long long q = apsi(g.n, g.L, 2, s2, i0, j, k);
        const V4 o0 = ld4(f.psiH[2][0] + q), o1 = ld4(f.psiH[2][1] + q);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            pzx.v[m] = o0.v[m] + (b * o0.v[m] + a * dEy_dz[m]);
            pzy.v[m] = o1.v[m] + (b * o1.v[m] + a * dEx_dz[m]);
        }
        st4(f.psiH[2][0] + q, pzx);
        st4(f.psiH[2][1] + q, pzy);
    }
#pragma unroll
    for (int m = 0; m < 4; m++) {
        hx.v[m] -= g.cH * (ky * dEz_dy[m] + pyx.v[m] - kz * dEy_dz[m] - pzx.v[m]);
        hy.v[m] -= g.cH * (kz * dEx_dz[m] + pzy.v[m] - kx[m] * dEz_dx[m] - pxy.v[m]);
        hz.v[m] -= g.cH * (kx[m] * dEy_dx[m] + pxz.v[m] - ky * dEx_dy[m] - pyz.v[m]);
    }
    st4(f.H[0] + e, hx);
    st4(f.H[1] + e, hy);
    st4(f.H[2] + e, hz);
}

// Eq. 6 on the design edges among the four, then Eq. 8, for component c of
// cells e..e+3 at plane k; held cells (upd false) keep E, J and psi.
__device__ __forceinline__ void fwd_ampere4(const AGrid<float> &g, const AState<float> &f, int c, long long e, int k,
                                            long long nr, const float curl[4], const float js[4], const bool upd[4]) {
    V4 E = ld4(f.E[c] + e);
    if (k >= g.ks0 && k < g.ks1) {
        const int4 s4 = *reinterpret_cast<const int4 *>(f.slot[c] + e);
        const int sl[4] = {s4.x, s4.y, s4.z, s4.w};
        const long long ne = f.soff[3];
#pragma unroll
        for (int m = 0; m < 4; m++) {
            float jp = 0.f;
            if (sl[m] >= 0 && upd[m]) {
                const float j0 = f.J[c][e + m];
                const long long row = nr * ne + sl[m];
                f.stE[row] = E.v[m];
                f.stJ[row] = j0;
                jp = j0 + (g.kJm1 * j0 + f.beta[sl[m]] * E.v[m]);
                f.J[c][e + m] = jp;
            }
            if (upd[m]) E.v[m] = E.v[m] + g.cE * (curl[m] - jp - js[m]);
        }
    } else {
#pragma unroll
        for (int m = 0; m < 4; m++)
            if (upd[m]) E.v[m] = E.v[m] + g.cE * (curl[m] - js[m]);
    }
    st4(f.E[c] + e, E);
}

// psi update of one axis for the four cells (profiles per cell along x,
// per row or plane along y and z); held cells keep their psi.  Returns the
// new psi values in p and the 1/kappa factors in kap.
__device__ __forceinline__ void psi4(float *psi, long long q, const float *bb, const float *aa, const float *ik, int x0,
                                     bool per_cell, const float d[4], const bool upd[4], float p[4], float kap[4]) {
    V4 o = ld4(psi + q);
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const int x = per_cell ? x0 + m : x0;
        const float b = bb[x], a = aa[x];
        kap[m] = ik[x];
        p[m] = o.v[m] + (b * o.v[m] + a * d[m]);
        if (upd[m]) o.v[m] = p[m];
    }
    st4(psi + q, o);
}

__global__ void __launch_bounds__(256) k_fwd_E4(AGrid<float> g, AState<float> f, Bunch bu, double dt) {
    pdl_wait();
    pdl_release();
    const long long n = *f.n, nr = n % f.seg;
    (void)dt;
    int i0, j, k;
    if (!group_of(g, i0, j, k)) return;
    const int nx = g.n[0], ny = g.n[1];
    const long long sy = nx, sz = (long long)nx * ny, e = k * sz + j * sy + i0;
    const bool fx0 = i0 == 0, fy = j == 0, fz = k == 0;
    const long long ojm = j > 0 ? sy : 0, okm = k > 0 ? sz : 0;
    const V4 hx = ld4(f.H[0] + e), hy = ld4(f.H[1] + e), hz = ld4(f.H[2] + e);
    const float hz_im = f.H[2][e - (i0 > 0 ? 1 : 0)], hy_im = f.H[1][e - (i0 > 0 ? 1 : 0)];
    const int s0 = aslab(g.L, nx, i0), s1 = aslab(g.L, ny, j), s2 = aslab(g.L, g.n[2], k);
    const float rx = g.r[0], ry = g.r[1], rz = g.r[2];
    const float zero[4] = {0.f, 0.f, 0.f, 0.f};
    // component c: curl = k1 d1 + p1 - k2 d2 - p2 over its two transverse axes
    if (!(fy || fz)) {  // Ex: d1 = dHz/dy (psi_E[1][1]), d2 = dHy/dz (psi_E[2][0])
        const V4 hz_jm = ld4(f.H[2] + e - ojm), hy_km = ld4(f.H[1] + e - okm);
        const bool upd[4] = {true, true, true, true};
        float d1[4], d2[4], k1[4] = {1.f, 1.f, 1.f, 1.f}, k2[4] = {1.f, 1.f, 1.f, 1.f}, p1[4] = {0.f, 0.f, 0.f, 0.f},
              p2[4] = {0.f, 0.f, 0.f, 0.f}, curl[4], js[4];
#pragma unroll
        for (int m = 0; m < 4; m++) {
            d1[m] = (hz.v[m] - hz_jm.v[m]) * ry;
            d2[m] = (hy.v[m] - hy_km.v[m]) * rz;
            js[m] = bunch_jx<float>(bu, i0 + m, j, k, n);
        }
        if (s1 >= 0) psi4(f.psiE[1][1], apsi(g.n, g.L, 1, s1, i0, j, k), f.bE[1], f.aE[1], f.ikE[1], j, false, d1, upd, p1, k1);
        if (s2 >= 0) psi4(f.psiE[2][0], apsi(g.n, g.L, 2, s2, i0, j, k), f.bE[2], f.aE[2], f.ikE[2], k, false, d2, upd, p2, k2);
#pragma unroll
        for (int m = 0; m < 4; m++) curl[m] = k1[m] * d1[m] + p1[m] - k2[m] * d2[m] - p2[m];
        fwd_ampere4(g, f, 0, e, k, nr, curl, js, upd);
    }
    if (!fz) {  // Ey: d1 = dHx/dz (psi_E[2][1]), d2 = dHz/dx (psi_E[0][0]); cell 0 held on the x face
        const V4 hx_km = ld4(f.H[0] + e - okm);
        const bool upd[4] = {!fx0, true, true, true};
        float d1[4], d2[4], k1[4] = {1.f, 1.f, 1.f, 1.f}, k2[4] = {1.f, 1.f, 1.f, 1.f}, p1[4] = {0.f, 0.f, 0.f, 0.f},
              p2[4] = {0.f, 0.f, 0.f, 0.f}, curl[4];
#pragma unroll
        for (int m = 0; m < 4; m++) {
            d1[m] = (hx.v[m] - hx_km.v[m]) * rz;
            d2[m] = (hz.v[m] - (m > 0 ? hz.v[m - 1] : hz_im)) * rx;
        }
        if (s2 >= 0) psi4(f.psiE[2][1], apsi(g.n, g.L, 2, s2, i0, j, k), f.bE[2], f.aE[2], f.ikE[2], k, false, d1, upd, p1, k1);
        if (s0 >= 0) psi4(f.psiE[0][0], apsi(g.n, g.L, 0, s0, i0, j, k), f.bE[0], f.aE[0], f.ikE[0], i0, true, d2, upd, p2, k2);
#pragma unroll
        for (int m = 0; m < 4; m++) curl[m] = k1[m] * d1[m] + p1[m] - k2[m] * d2[m] - p2[m];
        fwd_ampere4(g, f, 1, e, k, nr, curl, zero, upd);
    }
    if (!fy) {  // Ez: d1 = dHy/dx (psi_E[0][1]), d2 = dHx/dy (psi_E[1][0]); cell 0 held on the x face
        const V4 hx_jm = ld4(f.H[0] + e - ojm);
        const bool upd[4] = {!fx0, true, true, true};
        float d1[4], d2[4], k1[4] = {1.f, 1.f, 1.f, 1.f}, k2[4] = {1.f, 1.f, 1.f, 1.f}, p1[4] = {0.f, 0.f, 0.f, 0.f},
              p2[4] = {0.f, 0.f, 0.f, 0.f}, curl[4];
#pragma unroll
        for (int m = 0; m < 4; m++) {
            d1[m] = (hy.v[m] - (m > 0 ? hy.v[m - 1] : hy_im)) * rx;
            d2[m] = (hx.v[m] - hx_jm.v[m]) * ry;
        }
        if (s0 >= 0) psi4(f.psiE[0][1], apsi(g.n, g.L, 0, s0, i0, j, k), f.bE[0], f.aE[0], f.ikE[0], i0, true, d1, upd, p1, k1);
        if (s1 >= 0) psi4(f.psiE[1][0], apsi(g.n, g.L, 1, s1, i0, j, k), f.bE[1], f.aE[1], f.ikE[1], j, false, d2, upd, p2, k2);
#pragma unroll
        for (int m = 0; m < 4; m++) curl[m] = k1[m] * d1[m] + p1[m] - k2[m] * d2[m] - p2[m];
        fwd_ampere4(g, f, 2, e, k, nr, curl, zero, upd);
    }
}

// transposed psi_H recursion of one axis: p = psi + sg cH l (l the lambda_H
// the psi term enters), A = sg cH kappa^-1 l + a p, psi <- (1 + b) p
__device__ __forceinline__ void psiH4_adj(float *psi, long long q, float b1, float a, float ik, float sg, float cH,
                                          const float l[4], float A[4]) {
    V4 o = ld4(psi + q);
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const float p = o.v[m] + sg * cH * l[m];
        A[m] = sg * cH * ik * l[m] + a * p;
        o.v[m] = b1 * p;
    }
    st4(psi + q, o);
}

__global__ void __launch_bounds__(256) k_adj_H4(AGrid<float> g, AState<float> f) {
    pdl_wait();
    pdl_release();
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0) *f.n -= 1;
    int i0, j, k;
    if (!group_of(g, i0, j, k)) return;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long sy = nx, sz = (long long)nx * ny, e = k * sz + j * sy + i0;
    const V4 LX = ld4(f.lH[0] + e), LY = ld4(f.lH[1] + e), LZ = ld4(f.lH[2] + e);
    const float cH = g.cH, rx = g.r[0], ry = g.r[1], rz = g.r[2];
    // adjoints of the six differences (forward differences of E)
    float Azy[4], Ayz[4], Axz[4], Azx[4], Ayx[4], Axy[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        Azy[m] = -cH * LX.v[m]; Ayz[m] = cH * LX.v[m];
        Axz[m] = -cH * LY.v[m]; Azx[m] = cH * LY.v[m];
        Ayx[m] = -cH * LZ.v[m]; Axy[m] = cH * LZ.v[m];
    }
    const int s0 = aslab(g.L, nx, i0), s1 = aslab(g.L, ny, j), s2 = aslab(g.L, nz, k);
    if (s0 >= 0) {  // per-cell profiles along x
        const long long q = apsi(g.n, g.L, 0, s0, i0, j, k);
        V4 o0 = ld4(f.lpsiH[0][0] + q), o1 = ld4(f.lpsiH[0][1] + q);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const float a = f.aH[0][i0 + m], kk = f.ikH[0][i0 + m], b1 = 1.f + f.bH[0][i0 + m];
            const float pxy = o0.v[m] + cH * LY.v[m], pxz = o1.v[m] - cH * LZ.v[m];
            Azx[m] = cH * kk * LY.v[m] + a * pxy;
            Ayx[m] = -cH * kk * LZ.v[m] + a * pxz;
            o0.v[m] = b1 * pxy;
            o1.v[m] = b1 * pxz;
        }
        st4(f.lpsiH[0][0] + q, o0);
        st4(f.lpsiH[0][1] + q, o1);
    }
    if (s1 >= 0) {
        const long long q = apsi(g.n, g.L, 1, s1, i0, j, k);
        const float a = f.aH[1][j], kk = f.ikH[1][j], b1 = 1.f + f.bH[1][j];
        psiH4_adj(f.lpsiH[1][0], q, b1, a, kk, 1.f, cH, LZ.v, Axy);
        psiH4_adj(f.lpsiH[1][1], q, b1, a, kk, -1.f, cH, LX.v, Azy);
    }
    if (s2 >= 0) {
        const long long q = apsi(g.n, g.L, 2, s2, i0, j, k);
        const float a = f.aH[2][k], kk = f.ikH[2][k], b1 = 1.f + f.bH[2][k];
        psiH4_adj(f.lpsiH[2][0], q, b1, a, kk, 1.f, cH, LX.v, Ayz);
        psiH4_adj(f.lpsiH[2][1], q, b1, a, kk, -1.f, cH, LY.v, Axz);
    }
    // d = (E[e' + e_a] - E[e']) r, E beyond the high face zero: the own cell
    // gets -r A, the cell at +e_a gets +r A
    float own[3][4], e2_yp[4], e0_yp[4], e1_zp[4], e0_zp[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        own[2][m] = -ry * Azy[m] - rx * Azx[m] + (m > 0 ? rx * Azx[m - 1] : 0.f);
        own[1][m] = -rz * Ayz[m] - rx * Ayx[m] + (m > 0 ? rx * Ayx[m - 1] : 0.f);
        own[0][m] = -rz * Axz[m] - ry * Axy[m];
        e2_yp[m] = ry * Azy[m];
        e0_yp[m] = ry * Axy[m];
        e1_zp[m] = rz * Ayz[m];
        e0_zp[m] = rz * Axz[m];
    }
    add4(f.lE[0] + e, V4{{own[0][0], own[0][1], own[0][2], own[0][3]}});
    add4(f.lE[1] + e, V4{{own[1][0], own[1][1], own[1][2], own[1][3]}});
    add4(f.lE[2] + e, V4{{own[2][0], own[2][1], own[2][2], own[2][3]}});
    if (j + 1 < ny) {
        add4(f.lE[2] + e + sy, V4{{e2_yp[0], e2_yp[1], e2_yp[2], e2_yp[3]}});
        add4(f.lE[0] + e + sy, V4{{e0_yp[0], e0_yp[1], e0_yp[2], e0_yp[3]}});
    }
    if (k + 1 < nz) {
        add4(f.lE[1] + e + sz, V4{{e1_zp[0], e1_zp[1], e1_zp[2], e1_zp[3]}});
        add4(f.lE[0] + e + sz, V4{{e0_zp[0], e0_zp[1], e0_zp[2], e0_zp[3]}});
    }
    if (i0 + 4 < nx) {
        atomicAdd(f.lE[2] + e + 4, rx * Azx[3]);
        atomicAdd(f.lE[1] + e + 4, rx * Ayx[3]);
    }
}

// ------------------------------------------------------------------ host --
struct AdjBase {
    virtual ~AdjBase() {}
    virtual int forward(const double *mask, double wp, double gamma, double *loss) = 0;
    virtual int backward(double *dmask, double *dwp, double *dgamma) = 0;
    long long nmask = 0;
};

template <typename T>
struct AdjSim : AdjBase {
    pic_adj_config cfg{};
    AGrid<T> g{};
    AState<T> f{};
    Bunch bu{};
    Probe pr{};
    long long N = 0, ne = 0;
    std::vector<void *> allocs;
    std::vector<long long> eidx_h;       // per slot: edge index
    std::vector<int> comp_h;             // per slot: component
    std::vector<T> beta_h;
    std::vector<double> mbar_h;          // per slot: mean mask over its four cells (last forward)
    std::vector<std::array<long long, 4>> cells_h;  // per slot: its four cells as mask indices (-1: outside)
    double *d_F = nullptr;
    double F[2] = {0, 0};
    cudaStream_t stream = nullptr;
    bool use4 = false;  // FP32 with four-cell groups (nx and the CPML width multiples of 4)
    static constexpr int GRAPH_STEPS = 64;  // steps per captured graph (forward and backward)
    cudaGraphExec_t gfwd = nullptr, gbwd = nullptr, grec = nullptr;  // forward, backward, recompute
    double wp_last = 0, gamma_last = 0;
    bool have_forward = false;
    // checkpoint mode (flags bit 1): the field state every C steps; each
    // segment's E^n, J^n are recomputed from its checkpoint during the backward
    bool ckpt = false;
    long long C = 0, K = 1;                               // segment length, segments
    std::vector<std::pair<T *, size_t>> state;            // the forward state arrays (E, H, J, psi)
    size_t state_elems = 0;
    T *ckbuf = nullptr;                                   // checkpoints 1..K-1 (0 is the zero state)
    double *d_Fr = nullptr;                               // probe sum of the recomputed steps (discarded)

    ~AdjSim() override {
        if (stream) cudaStreamSynchronize(stream);
        if (gfwd) cudaGraphExecDestroy(gfwd);
        if (gbwd) cudaGraphExecDestroy(gbwd);
        if (grec) cudaGraphExecDestroy(grec);
        for (void *p : allocs) cudaFree(p);
        if (stream) cudaStreamDestroy(stream);
    }

    template <typename P>
    int take(P **out, size_t count) {
        void *p = nullptr;
        if (cudaMalloc(&p, count * sizeof(P) + 16) != cudaSuccess)
            return set_last_error(PIC_ERR_OOM, "adjoint: cudaMalloc of %zu bytes failed", count * sizeof(P));
        allocs.push_back(p);
        *out = static_cast<P *>(p);
        return PIC_OK;
    }

    void profile(int a, double pos, double &b, double &aa, double &ik) const {
        const double L = cfg.cpml_cells, n = (double)g.n[a];
        double rho = 0.0;
        if (pos < L) rho = L - pos;
        if (pos > n - L) rho = std::max(rho, pos - (n - L));
        if (rho <= 0.0) { b = 0.0; aa = 0.0; ik = 1.0; return; }
        const double eta0 = std::sqrt(cfg.mu0 / cfg.eps0);
        const double x = rho / L, xm = std::pow(x, cfg.cpml_order);
        const double sigma = cfg.cpml_sigma_fac * (cfg.cpml_order + 1.0) / (eta0 * cfg.dx) * xm;
        const double kappa = 1.0 + (cfg.cpml_kappa_max - 1.0) * xm;
        const double alpha = cfg.cpml_alpha_max * (1.0 - x);
        b = std::expm1(-(sigma / kappa + alpha) * cfg.dt / cfg.eps0);
        const double den = sigma * kappa + kappa * kappa * alpha;
        aa = (sigma > 0.0 && den > 0.0) ? sigma * b / den : 0.0;
        ik = 1.0 / kappa;
    }

    int create(const pic_adj_config *c) {
        cfg = *c;
        for (int a = 0; a < 3; a++) g.n[a] = (int)(a == 0 ? c->nx : a == 1 ? c->ny : c->nz);
        g.L = c->cpml_cells;
        for (int a = 0; a < 3; a++) g.r[a] = (T)(1.0 / c->dx);
        g.cH = (T)(c->dt / c->mu0);
        g.cE = (T)(c->dt / c->eps0);
        N = (long long)g.n[0] * g.n[1] * g.n[2];
        const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
        nmask = (long long)nx * ny * (c->design_k1 - c->design_k0);
        // design edges: any of the four cells around the edge inside the slab
        // (cells beyond a face are clamped to the face, as for the materials)
        auto cell_mask_index = [&](int i, int j, int k) -> long long {
            i = std::min(std::max(i, 0), nx - 1);
            j = std::min(std::max(j, 0), ny - 1);
            k = std::min(std::max(k, 0), nz - 1);
            if (k < c->design_k0 || k >= c->design_k1) return -1;
            return ((long long)(k - c->design_k0) * ny + j) * nx + i;
        };
        use4 = std::is_same<T, float>::value && nx % 4 == 0 && g.L % 4 == 0 && !(c->flags & 1);
        g.ks0 = std::max(0, (int)c->design_k0 - 1);
        g.ks1 = std::min(nz, (int)c->design_k1 + 1);
        std::vector<int> slot_h[3];
        long long soff[4] = {0, 0, 0, 0};
        for (int comp = 0; comp < 3; comp++) {
            slot_h[comp].assign((size_t)N, -1);
            const int a1 = (comp + 1) % 3, a2 = (comp + 2) % 3;
            const int klo = g.ks0, khi = g.ks1;
            for (int k = klo; k < khi; k++)
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        std::array<long long, 4> cl;
                        bool any = false;
                        int t = 0;
                        for (int s1 = -1; s1 <= 0; s1++)
                            for (int s2 = -1; s2 <= 0; s2++) {
                                int p3[3] = {i, j, k};
                                p3[a1] += s1;
                                p3[a2] += s2;
                                cl[t] = cell_mask_index(p3[0], p3[1], p3[2]);
                                any = any || cl[t] >= 0;
                                t++;
                            }
                        if (!any) continue;
                        const long long e = ((long long)k * ny + j) * nx + i;
                        slot_h[comp][(size_t)e] = (int)eidx_h.size();
                        eidx_h.push_back(e);
                        comp_h.push_back(comp);
                        cells_h.push_back(cl);
                    }
            soff[comp + 1] = (long long)eidx_h.size();
        }
        ne = (long long)eidx_h.size();
        ckpt = (c->flags & 2) != 0;
        if (ckpt) {  // segments of 64 * ceil(sqrt(nsteps) / 64) steps
            const long long r = (long long)std::ceil(std::sqrt((double)c->nsteps) / GRAPH_STEPS);
            C = GRAPH_STEPS * std::max(1LL, r);
            K = (c->nsteps + C - 1) / C;
        } else {
            C = c->nsteps;
            K = 1;
        }
        f.seg = C;
        const size_t per_step = (size_t)ne * 2 * sizeof(T);
        if (per_step && (size_t)C > ((size_t)1 << 40) / per_step)
            return set_last_error(PIC_ERR_OOM, "adjoint storage of %lld steps x %lld edges is too large",
                                  (long long)C, ne);
        // device arrays
        int rc = 0;
        for (int a = 0; a < 3 && !rc; a++) {
            rc = rc ? rc : take(&f.E[a], N);
            rc = rc ? rc : take(&f.H[a], N);
            rc = rc ? rc : take(&f.J[a], N);
            rc = rc ? rc : take(&f.lE[a], N);
            rc = rc ? rc : take(&f.lH[a], N);
            rc = rc ? rc : take(&f.lJ[a], N);
            const size_t slab = (size_t)(N / g.n[a]) * 2 * g.L;
            for (int s = 0; s < 2 && !rc; s++) {
                rc = rc ? rc : take(&f.psiH[a][s], slab);
                rc = rc ? rc : take(&f.psiE[a][s], slab);
                rc = rc ? rc : take(&f.lpsiH[a][s], slab);
                rc = rc ? rc : take(&f.lpsiE[a][s], slab);
            }
        }
        T *prof[3][6];
        int *slot_d[3];
        long long *eidx_d = nullptr;
        T *beta_d = nullptr;
        for (int a = 0; a < 3 && !rc; a++) {
            for (int q6 = 0; q6 < 6 && !rc; q6++) rc = take(&prof[a][q6], g.n[a]);
            rc = rc ? rc : take(&slot_d[a], N);
        }
        rc = rc ? rc : take(&eidx_d, ne + 1);
        rc = rc ? rc : take(&beta_d, ne + 1);
        rc = rc ? rc : take(&f.gb, ne + 1);
        rc = rc ? rc : take(&f.gk, ne + 1);
        rc = rc ? rc : take(&f.stE, (size_t)ne * C + 1);
        rc = rc ? rc : take(&f.stJ, (size_t)ne * C + 1);
        rc = rc ? rc : take(&d_F, 2);
        rc = rc ? rc : take(&d_Fr, 2);
        if (!rc) {
            for (int a = 0; a < 3; a++) {
                state.emplace_back(f.E[a], (size_t)N);
                state.emplace_back(f.H[a], (size_t)N);
                state.emplace_back(f.J[a], (size_t)N);
                const size_t slab = (size_t)(N / g.n[a]) * 2 * g.L;
                for (int s2 = 0; s2 < 2; s2++) {
                    state.emplace_back(f.psiH[a][s2], slab);
                    state.emplace_back(f.psiE[a][s2], slab);
                }
            }
            state_elems = 0;
            for (auto &st : state) state_elems += st.second;
            if (ckpt && K > 1) rc = take(&ckbuf, state_elems * (size_t)(K - 1));
        }
        rc = rc ? rc : take(&f.n, 1);
        double *gx64 = nullptr, *gyz64 = nullptr;
        float *gx32 = nullptr, *gyz32 = nullptr;
        rc = rc ? rc : take(&gx64, (size_t)c->nsteps * nx);
        rc = rc ? rc : take(&gx32, (size_t)c->nsteps * nx);
        rc = rc ? rc : take(&gyz64, (size_t)nz * ny);
        rc = rc ? rc : take(&gyz32, (size_t)nz * ny);
        if (rc) return rc;
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess)
            return set_last_error(PIC_ERR_CUDA, "adjoint: stream creation failed");
        for (int a = 0; a < 3; a++) {
            std::vector<T> pf[6];
            for (auto &v : pf) v.resize(g.n[a]);
            for (int x = 0; x < g.n[a]; x++) {
                double b, aa, ik;
                profile(a, (double)x, b, aa, ik);
                pf[0][x] = (T)b; pf[1][x] = (T)aa; pf[2][x] = (T)ik;
                profile(a, x + 0.5, b, aa, ik);
                pf[3][x] = (T)b; pf[4][x] = (T)aa; pf[5][x] = (T)ik;
            }
            for (int q6 = 0; q6 < 6; q6++)
                if (cudaMemcpy(prof[a][q6], pf[q6].data(), g.n[a] * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
                    return set_last_error(PIC_ERR_CUDA, "adjoint: profile upload failed");
            f.bE[a] = prof[a][0]; f.aE[a] = prof[a][1]; f.ikE[a] = prof[a][2];
            f.bH[a] = prof[a][3]; f.aH[a] = prof[a][4]; f.ikH[a] = prof[a][5];
            if (cudaMemcpy(slot_d[a], slot_h[a].data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
                return set_last_error(PIC_ERR_CUDA, "adjoint: edge map upload failed");
            f.slot[a] = slot_d[a];
        }
        if (ne && cudaMemcpy(eidx_d, eidx_h.data(), (size_t)ne * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess)
            return set_last_error(PIC_ERR_CUDA, "adjoint: edge list upload failed");
        f.eidx = eidx_d;
        f.beta = beta_d;
        for (int q4 = 0; q4 < 4; q4++) f.soff[q4] = soff[q4];
        // bunch: the two factors of the Gaussian current on every Ex edge
        {
            const double s = c->bunch_sigma, inv2s2 = 1.0 / (2.0 * s * s);
            const double qv_norm = c->bunch_q * c->bunch_v / std::pow(2.0 * M_PI * s * s, 1.5);
            std::vector<double> gx((size_t)c->nsteps * nx), gyz((size_t)nz * ny);
            for (long long n = 0; n < c->nsteps; n++) {
                const double xc = c->bunch_x0 + c->bunch_v * ((double)n + 0.5) * c->dt;
                for (int i = 0; i < nx; i++) {
                    const double x = (i + 0.5) * c->dx - xc;
                    gx[(size_t)n * nx + i] = std::exp(-x * x * inv2s2);
                }
            }
            for (int k = 0; k < nz; k++)
                for (int j = 0; j < ny; j++) {
                    const double y = j * c->dx - c->bunch_y0, z = k * c->dx - c->bunch_z0;
                    gyz[(size_t)k * ny + j] = qv_norm * std::exp(-(y * y + z * z) * inv2s2);
                }
            std::vector<float> gx_f(gx.begin(), gx.end()), gyz_f(gyz.begin(), gyz.end());
            if (cudaMemcpy(gx64, gx.data(), gx.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(gx32, gx_f.data(), gx_f.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(gyz64, gyz.data(), gyz.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(gyz32, gyz_f.data(), gyz_f.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
                return set_last_error(PIC_ERR_CUDA, "adjoint: bunch table upload failed");
            bu.gx64 = gx64; bu.gyz64 = gyz64; bu.gx32 = gx32; bu.gyz32 = gyz32;
            bu.nx = nx; bu.ny = ny; bu.nsteps = c->nsteps;
        }
        // probe stencil on the component's staggered lattice
        pr.comp = c->probe_comp;
        pr.omega = c->omega0;
        pr.dt = c->dt;
        for (int corner = 0; corner < 8; corner++) {
            long long idx = 0, stride = 1;
            double wt = 1.0;
            for (int a = 0; a < 3; a++) {
                const double sa = c->probe[a] / c->dx - (a == pr.comp ? 0.5 : 0.0);
                const double fl = std::floor(sa);
                const int bit = (corner >> a) & 1;
                const int ib = std::min(std::max((int)fl + bit, 0), g.n[a] - 1);
                wt *= bit ? (sa - fl) : 1.0 - (sa - fl);
                idx += (long long)ib * stride;
                stride *= g.n[a];
            }
            pr.idx[corner] = idx;
            pr.w[corner] = wt;
        }
        for (int a = 0; a < 3; a++) {  // index range of the corners along each axis
            long long stride = 1;
            for (int b = 0; b < a; b++) stride *= g.n[b];
            pr.lo[a] = g.n[a];
            pr.hi[a] = -1;
            for (int corner = 0; corner < 8; corner++) {
                const int x = (int)((pr.idx[corner] / stride) % g.n[a]);
                pr.lo[a] = std::min(pr.lo[a], x);
                pr.hi[a] = std::max(pr.hi[a], x);
            }
        }
        return PIC_OK;
    }

    void clear_forward() {
        for (auto &st : state) cudaMemsetAsync(st.first, 0, st.second * sizeof(T), stream);
        cudaMemsetAsync(d_F, 0, 2 * sizeof(double), stream);
        cudaMemsetAsync(f.n, 0xff, sizeof(long long), stream);  // -1: no step taken yet
    }
    // the forward state to or from checkpoint k (1..K-1)
    void save_state(long long k) {
        T *dst = ckbuf + state_elems * (size_t)(k - 1);
        for (auto &st : state) {
            cudaMemcpyAsync(dst, st.first, st.second * sizeof(T), cudaMemcpyDeviceToDevice, stream);
            dst += st.second;
        }
    }
    void load_state(long long k) {
        if (k == 0) {
            for (auto &st : state) cudaMemsetAsync(st.first, 0, st.second * sizeof(T), stream);
            return;
        }
        const T *src = ckbuf + state_elems * (size_t)(k - 1);
        for (auto &st : state) {
            cudaMemcpyAsync(st.first, src, st.second * sizeof(T), cudaMemcpyDeviceToDevice, stream);
            src += st.second;
        }
    }
    void clear_adjoint() {
        for (int a = 0; a < 3; a++) {
            cudaMemsetAsync(f.lE[a], 0, N * sizeof(T), stream);
            cudaMemsetAsync(f.lH[a], 0, N * sizeof(T), stream);
            cudaMemsetAsync(f.lJ[a], 0, N * sizeof(T), stream);
            const size_t slab = (size_t)(N / g.n[a]) * 2 * g.L;
            for (int s = 0; s < 2; s++) {
                cudaMemsetAsync(f.lpsiH[a][s], 0, slab * sizeof(T), stream);
                cudaMemsetAsync(f.lpsiE[a][s], 0, slab * sizeof(T), stream);
            }
        }
        cudaMemsetAsync(f.gb, 0, ne * sizeof(double), stream);
        cudaMemsetAsync(f.gk, 0, ne * sizeof(double), stream);
    }

    // 32 x 8 threads over (x, y), one plane z per grid layer
    static dim3 block3() { return dim3(32, 8, 1); }
    dim3 grid3() const { return dim3((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, g.n[2]); }
    // four-cell groups: 32 (or 16, when that divides the row and 32 does not) groups along x
    dim3 block4() const {
        const int groups = g.n[0] / 4;
        return (groups % 32 != 0 && groups % 16 == 0) ? dim3(16, 16, 1) : dim3(32, 8, 1);
    }
    dim3 grid4() const {
        const dim3 b = block4();
        return dim3((g.n[0] / 4 + b.x - 1) / b.x, (g.n[1] + b.y - 1) / b.y, g.n[2]);
    }

    T kJm1_captured = T(0);
    void drop_graphs() {
        if (gfwd) cudaGraphExecDestroy(gfwd);
        if (gbwd) cudaGraphExecDestroy(gbwd);
        if (grec) cudaGraphExecDestroy(grec);
        gfwd = gbwd = grec = nullptr;
    }
    void launch_forward_steps(int count) { launch_forward_steps(count, d_F); }
    // forward steps that add their probe terms to Fp
    void launch_forward_steps(int count, double *Fp) {
        const dim3 gr = grid3(), bl = block3();
        if constexpr (std::is_same<T, float>::value) {
            if (use4) {
                const dim3 g4 = grid4(), b4 = block4();
                for (int q = 0; q < count; q++) {
                    launch_pdl(k_fwd_H4, g4, b4, 0, stream, g, f, pr, Fp, bu, cfg.dt);
                    launch_pdl(k_fwd_E4, g4, b4, 0, stream, g, f, bu, cfg.dt);
                }
                return;
            }
        }
        for (int q = 0; q < count; q++) {
            launch_pdl(k_fwd_H<T>, gr, bl, 0, stream, g, f, pr, Fp, bu, cfg.dt);
            launch_pdl(k_fwd_E<T>, gr, bl, 0, stream, g, f, bu, cfg.dt);
        }
    }
    void launch_backward_steps(int count) {
        const dim3 gr = grid3(), bl = block3();
        if constexpr (std::is_same<T, float>::value) {
            if (use4) {
                const dim3 g4 = grid4(), b4 = block4();
                for (int q = 0; q < count; q++) {
                    launch_pdl(k_adj_E<T>, gr, bl, 0, stream, g, f, pr, (const double *)d_F);
                    launch_pdl(k_adj_H4, g4, b4, 0, stream, g, f);
                }
                return;
            }
        }
        for (int q = 0; q < count; q++) {
            launch_pdl(k_adj_E<T>, gr, bl, 0, stream, g, f, pr, (const double *)d_F);
            launch_pdl(k_adj_H<T>, gr, bl, 0, stream, g, f);
        }
    }
    // one block of GRAPH_STEPS steps from a graph captured on first use (the
    // step index lives in device memory, so one graph serves every block)
    // fwd: forward steps adding to Fp; else backward steps
    int run_block(bool fwd, cudaGraphExec_t &exec, double *Fp = nullptr) {
        if (!exec) {
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return set_last_error(PIC_ERR_CUDA, "adjoint: graph capture failed to start");
            if (fwd) launch_forward_steps(GRAPH_STEPS, Fp ? Fp : d_F);
            else launch_backward_steps(GRAPH_STEPS);
            cudaError_t e = cudaStreamEndCapture(stream, &graph);
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                exec = nullptr;
                return set_last_error(PIC_ERR_CUDA, "adjoint graph: %s", cudaGetErrorString(e));
            }
            if (fwd) kJm1_captured = g.kJm1;
        }
        if (cudaGraphLaunch(exec, stream) != cudaSuccess)
            return set_last_error(PIC_ERR_CUDA, "adjoint: graph launch failed");
        return PIC_OK;
    }

    int forward(const double *mask, double wp, double gamma, double *loss) override {
        if (!mask || !loss) return set_last_error(PIC_ERR_ARG, "NULL argument");
        if (!(wp >= 0.0) || !(gamma >= 0.0) || !std::isfinite(wp) || !std::isfinite(gamma))
            return set_last_error(PIC_ERR_ARG, "need finite wp >= 0 and gamma >= 0");
        for (long long q = 0; q < nmask; q++)
            if (!(mask[q] >= 0.0 && mask[q] <= 1.0)) return set_last_error(PIC_ERR_ARG, "mask[%lld] outside [0, 1]", q);
        const double dt = cfg.dt, c2 = 1.0 / (cfg.eps0 * cfg.mu0);
        if (!(c2 * dt * dt * 3.0 / (cfg.dx * cfg.dx) + 0.25 * wp * wp * dt * dt < 1.0))
            return set_last_error(PIC_ERR_CFL, "dt=%g violates the time-step bound with wp=%g", dt, wp);
        g.kJm1 = (T)(-2.0 * gamma * dt / (2.0 + gamma * dt));
        beta_h.resize(ne);
        mbar_h.resize(ne);
        for (long long q = 0; q < ne; q++) {
            double m = 0.0;
            for (int t = 0; t < 4; t++) m += cells_h[q][t] >= 0 ? mask[cells_h[q][t]] : 0.0;
            mbar_h[q] = 0.25 * m;
            beta_h[q] = (T)(2.0 * dt * cfg.eps0 * wp * wp * mbar_h[q] / (2.0 + gamma * dt));
        }
        if (ne && cudaMemcpy((void *)f.beta, beta_h.data(), ne * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
            return set_last_error(PIC_ERR_CUDA, "adjoint: bJ upload failed");
        // the bJ table above is uploaded by value into device memory, and the
        // kernels read kJ-1 from their arguments: graphs captured before
        // hold the old kJ-1, so they are rebuilt when gamma changes
        if (gfwd && kJm1_captured != g.kJm1) drop_graphs();
        clear_forward();
        long long done = 0;
        int rc = 0;
        while (done < cfg.nsteps && !rc) {
            if (ckpt && done > 0 && done % C == 0) save_state(done / C);  // the state after done steps
            if (cfg.nsteps - done >= GRAPH_STEPS) {
                rc = run_block(true, gfwd);
                done += GRAPH_STEPS;
            } else {
                launch_forward_steps((int)(cfg.nsteps - done));
                done = cfg.nsteps;
            }
        }
        if (rc) return rc;
        k_probe<T><<<1, 32, 0, stream>>>(f, pr, d_F);  // the last step's probe term
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(F, d_F, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return set_last_error(PIC_ERR_CUDA, "adjoint forward: %s", cudaGetErrorString(e));
        *loss = F[0] * F[0] + F[1] * F[1];
        wp_last = wp;
        gamma_last = gamma;
        have_forward = true;
        return PIC_OK;
    }

    int backward(double *dmask, double *dwp, double *dgamma) override {
        if (!have_forward) return set_last_error(PIC_ERR_STATE, "pic_adj_backward needs a forward run first");
        if (!dmask || !dwp || !dgamma) return set_last_error(PIC_ERR_ARG, "NULL argument");
        clear_adjoint();
        int rc = 0;
        // segments from the last to the first (one segment of all steps
        // unless in checkpoint mode, where each is first recomputed from its
        // checkpoint to refill the stored E^n, J^n)
        for (long long sgm = K - 1; sgm >= 0 && !rc; sgm--) {
            const long long start = sgm * C, len = std::min(C, (long long)cfg.nsteps - start);
            if (ckpt) {
                load_state(sgm);
                k_set_counter<<<1, 32, 0, stream>>>(f.n, start - 1);
                cudaMemsetAsync(d_Fr, 0, 2 * sizeof(double), stream);
                long long done = 0;
                while (done < len && !rc) {
                    if (len - done >= GRAPH_STEPS) {
                        rc = run_block(true, grec, d_Fr);
                        done += GRAPH_STEPS;
                    } else {
                        launch_forward_steps((int)(len - done), d_Fr);
                        done = len;
                    }
                }
            }
            k_set_counter<<<1, 32, 0, stream>>>(f.n, start + len);  // steps left at the segment's end
            long long left = len;
            while (left > 0 && !rc) {
                if (left >= GRAPH_STEPS) {
                    rc = run_block(false, gbwd);
                    left -= GRAPH_STEPS;
                } else {
                    launch_backward_steps((int)left);
                    left = 0;
                }
            }
        }
        if (rc) return rc;
        std::vector<double> gb(ne), gk(ne);
        cudaError_t e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess && ne) e = cudaMemcpy(gb.data(), f.gb, ne * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && ne) e = cudaMemcpy(gk.data(), f.gk, ne * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return set_last_error(PIC_ERR_CUDA, "adjoint backward: %s", cudaGetErrorString(e));
        // chain rule: bJ = 2 dt eps0 wp^2 mbar / (2 + gamma dt), kJ = (2 - gamma dt) / (2 + gamma dt)
        const double dt = cfg.dt, wp = wp_last, ga = gamma_last, den = 2.0 + ga * dt;
        const double dbeta_dm = 2.0 * dt * cfg.eps0 * wp * wp * 0.25 / den;  // per cell of the four
        const double dkJ_dga = -4.0 * dt / (den * den);
        for (long long q = 0; q < nmask; q++) dmask[q] = 0.0;
        double gwp = 0.0, gga = 0.0;
        for (long long q = 0; q < ne; q++) {
            for (int t = 0; t < 4; t++)
                if (cells_h[q][t] >= 0) dmask[cells_h[q][t]] += gb[q] * dbeta_dm;
            const double beta = 2.0 * dt * cfg.eps0 * wp * wp * mbar_h[q] / den;
            gwp += gb[q] * 2.0 * dt * cfg.eps0 * 2.0 * wp * mbar_h[q] / den;
            gga += gb[q] * (-beta * dt / den) + gk[q] * dkJ_dga;
        }
        *dwp = gwp;
        *dgamma = gga;
        return PIC_OK;
    }
};

}  // namespace
}  // namespace pic

struct pic_adj {
    pic::AdjBase *sim;
};

extern "C" {

int pic_adj_create(const pic_adj_config *c, pic_adj **out) {
    pic::NvtxRange nvtx_range("pic_adj_create");
    using namespace pic;
    set_last_error(PIC_OK, "%s", "");
    if (!out) return set_last_error(PIC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!c) return set_last_error(PIC_ERR_ARG, "config is NULL");
    if (c->precision != PIC_FP32 && c->precision != PIC_FP64) return set_last_error(PIC_ERR_ARG, "unknown precision");
    const int64_t n[3] = {c->nx, c->ny, c->nz};
    for (int a = 0; a < 3; a++)
        if (n[a] < 2 * (int64_t)c->cpml_cells + 4 || n[a] > 65535)
            return set_last_error(PIC_ERR_ARG, "axis %d: %lld cells do not hold two CPML slabs", a, (long long)n[a]);
    if (c->cpml_cells < 1) return set_last_error(PIC_ERR_ARG, "cpml_cells must be >= 1");
    if (!(c->dx > 0.0) || !(c->dt > 0.0) || !(c->eps0 > 0.0) || !(c->mu0 > 0.0))
        return set_last_error(PIC_ERR_ARG, "dx, dt, eps0, mu0 must be > 0");
    if (1.0 / (c->eps0 * c->mu0) * c->dt * c->dt * 3.0 / (c->dx * c->dx) >= 1.0)
        return set_last_error(PIC_ERR_CFL, "dt=%g violates the vacuum time-step bound", c->dt);
    if (c->design_k0 < 1 || c->design_k1 <= c->design_k0 || c->design_k1 > c->nz - 1)
        return set_last_error(PIC_ERR_ARG, "design slab [%lld, %lld) must lie inside the grid",
                              (long long)c->design_k0, (long long)c->design_k1);
    if (c->nsteps < 1) return set_last_error(PIC_ERR_ARG, "nsteps must be >= 1");
    if (c->nsteps * c->nx > (int64_t)1 << 28)
        return set_last_error(PIC_ERR_ARG, "nsteps x nx = %lld is above 2^28", (long long)(c->nsteps * c->nx));
    if (c->probe_comp < 0 || c->probe_comp > 2) return set_last_error(PIC_ERR_ARG, "probe_comp must be 0..2");
    for (int a = 0; a < 3; a++) {
        const double xi = c->probe[a] / c->dx;
        if (!(xi >= 1.0 && xi < n[a] - 1.0)) return set_last_error(PIC_ERR_ARG, "probe outside the grid interior");
    }
    if (!(c->bunch_sigma > 0.0)) return set_last_error(PIC_ERR_ARG, "bunch_sigma must be > 0");
    pic_adj *h = new pic_adj{nullptr};
    int rc;
    if (c->precision == PIC_FP64) {
        auto *s = new AdjSim<double>();
        h->sim = s;
        rc = s->create(c);
    } else {
        auto *s = new AdjSim<float>();
        h->sim = s;
        rc = s->create(c);
    }
    if (rc) {
        delete h->sim;
        delete h;
        return rc;
    }
    *out = h;
    return PIC_OK;
}

int pic_adj_mask_size(const pic_adj *a, int64_t *n) {
    pic::set_last_error(PIC_OK, "%s", "");
    if (!a || !n) return pic::set_last_error(PIC_ERR_ARG, "NULL argument");
    *n = a->sim->nmask;
    return PIC_OK;
}

int pic_adj_forward(pic_adj *a, const double *mask, double wp, double gamma, double *loss) {
    pic::NvtxRange nvtx_range("pic_adj_forward");
    pic::set_last_error(PIC_OK, "%s", "");
    if (!a) return pic::set_last_error(PIC_ERR_ARG, "NULL handle");
    return a->sim->forward(mask, wp, gamma, loss);
}

int pic_adj_backward(pic_adj *a, double *dmask, double *dwp, double *dgamma) {
    pic::NvtxRange nvtx_range("pic_adj_backward");
    pic::set_last_error(PIC_OK, "%s", "");
    if (!a) return pic::set_last_error(PIC_ERR_ARG, "NULL handle");
    return a->sim->backward(dmask, dwp, dgamma);
}

int pic_adj_destroy(pic_adj *a) {
    pic::NvtxRange nvtx_range("pic_adj_destroy");
    pic::set_last_error(PIC_OK, "%s", "");
    if (!a) return PIC_OK;
    delete a->sim;
    delete a;
    return PIC_OK;
}

}  // extern "C"
