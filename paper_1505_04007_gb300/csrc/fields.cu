// fields.cu -- Yee curl updates: the magnetic half step (vacuum Yee, Sec. II
// last paragraph) and the fused Drude-ADE + Ampere electric step (Eq. 6 then
// Eq. 8), each with the convolutional-PML terms inside the absorbing slabs.
//
// One thread per cell; x is the fastest index so a warp reads 32 consecutive
// floats/doubles of each array.  Forward (H) and backward (E) neighbours in
// y and z are re-reads of rows that neighbouring warps of the same block
// load, so they are served from L1/L2.
#include "pic_internal.cuh"

namespace pic {

template <typename T>
__device__ __forceinline__ int slab_pos(const Grid<T> &g, int a, int x) {
    if (!g.cpml[a]) return -1;
    if (x < g.L) return x;
    if (x >= g.n[a] - g.L) return x - (g.n[a] - 2 * g.L);
    return -1;
}

template <typename T>
__device__ __forceinline__ long long psi_at(const Grid<T> &g, int a, int s, int i, int j, int k) {
    const long long L2 = 2 * g.L;
    if (a == 0) return ((long long)k * g.n[1] + j) * L2 + s;
    if (a == 1) return ((long long)k * L2 + s) * g.n[0] + i;
    return ((long long)s * g.n[1] + j) * g.n[0] + i;
}

template <typename T>
__global__ void __launch_bounds__(256) k_update_H(Grid<T> g, Fields<T> f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (i >= nx || j >= ny || k >= nz) return;
    const long long sy = nx, sz = (long long)nx * ny;
    const long long e = k * sz + j * sy + i;

    // forward neighbour offsets; -1 marks "beyond a non-periodic face" (E = 0 there)
    long long oip = 1, ojp = sy, okp = sz;
    bool hip = true, hjp = true, hkp = true;
    if (i + 1 == nx) { if (g.per[0]) oip = -(long long)(nx - 1); else hip = false; }
    if (j + 1 == ny) { if (g.per[1]) ojp = -(long long)(ny - 1) * sy; else hjp = false; }
    if (k + 1 == nz) { if (g.per[2]) okp = -(long long)(nz - 1) * sz; else hkp = false; }

    // Clear the free current the previous step deposited in this tile (it
    // stays readable between steps; the deposit of this step refills it).
    const long long step = *f.step;
    const long long t = ((long long)(k / TILE_Z) * g.nt[1] + j / TILE_Y) * g.nt[0] + i / TILE_X;
    if (step > 0 && f.jf_flag[t] == (int)step) {
#pragma unroll
        for (int c = 0; c < 3; c++) f.Jf[c][e] = T(0);
    }

    const T *Ex = f.E[0], *Ey = f.E[1], *Ez = f.E[2];
    const T ex = Ex[e], ey = Ey[e], ez = Ez[e];
    const T zero = T(0);
    const T dEz_dy = ((hjp ? Ez[e + ojp] : zero) - ez) * g.r[1];
    const T dEy_dz = ((hkp ? Ey[e + okp] : zero) - ey) * g.r[2];
    const T dEx_dz = ((hkp ? Ex[e + okp] : zero) - ex) * g.r[2];
    const T dEz_dx = ((hip ? Ez[e + oip] : zero) - ez) * g.r[0];
    const T dEy_dx = ((hip ? Ey[e + oip] : zero) - ey) * g.r[0];
    const T dEx_dy = ((hjp ? Ex[e + ojp] : zero) - ex) * g.r[1];

    T kx = T(1), ky = T(1), kz = T(1);
    T pxy = zero, pxz = zero, pyz = zero, pyx = zero, pzx = zero, pzy = zero;
    const int s0 = slab_pos(g, 0, i), s1 = slab_pos(g, 1, j), s2 = slab_pos(g, 2, k);
    if (s0 >= 0) {
        const T b = f.bH[0][i], a = f.aH[0][i];
        kx = f.ikH[0][i];
        const long long q = psi_at(g, 0, s0, i, j, k);
        pxy = f.psiH[0][0][q] + (b * f.psiH[0][0][q] + a * dEz_dx); f.psiH[0][0][q] = pxy;  // Hy's d/dx
        pxz = f.psiH[0][1][q] + (b * f.psiH[0][1][q] + a * dEy_dx); f.psiH[0][1][q] = pxz;  // Hz's d/dx
    }
    if (s1 >= 0) {
        const T b = f.bH[1][j], a = f.aH[1][j];
        ky = f.ikH[1][j];
        const long long q = psi_at(g, 1, s1, i, j, k);
        pyz = f.psiH[1][0][q] + (b * f.psiH[1][0][q] + a * dEx_dy); f.psiH[1][0][q] = pyz;  // Hz's d/dy
        pyx = f.psiH[1][1][q] + (b * f.psiH[1][1][q] + a * dEz_dy); f.psiH[1][1][q] = pyx;  // Hx's d/dy
    }
    if (s2 >= 0) {
        const T b = f.bH[2][k], a = f.aH[2][k];
        kz = f.ikH[2][k];
        const long long q = psi_at(g, 2, s2, i, j, k);
        pzx = f.psiH[2][0][q] + (b * f.psiH[2][0][q] + a * dEy_dz); f.psiH[2][0][q] = pzx;  // Hx's d/dz
        pzy = f.psiH[2][1][q] + (b * f.psiH[2][1][q] + a * dEx_dz); f.psiH[2][1][q] = pzy;  // Hy's d/dz
    }
    const T cx = ky * dEz_dy + pyx - kz * dEy_dz - pzx;
    const T cy = kz * dEx_dz + pzy - kx * dEz_dx - pxy;
    const T cz = kx * dEy_dx + pxz - ky * dEx_dy - pyz;
    f.H[0][e] -= g.cH * cx;
    f.H[1][e] -= g.cH * cy;
    f.H[2][e] -= g.cH * cz;
}

// Eq. 6 on metal edges, then Eq. 8 without the free current (k_jf_apply
// subtracts that once the deposit of the step is complete).
template <typename T>
__device__ __forceinline__ void ampere(const Fields<T> &f, int c, long long e, T curl) {
    const int cls = f.ecls[c][e];
    T E = f.E[c][e];
    T jp = T(0);
    if (f.cls_metal[cls]) {
        // Eq. 6 written as an increment, J += (kJ-1) J + bJ E: the decay factor
        // kJ = (2-g dt)/(2+g dt) sits within g dt of 1, so kJ-1 (precomputed in
        // FP64) keeps the collision rate exact in FP32 where kJ itself would not.
        const T j0 = f.Jp[c][e];
        jp = j0 + (f.cls_kJm1[cls] * j0 + f.cls_bJ[cls] * E);
        f.Jp[c][e] = jp;
    }
    f.E[c][e] = E + f.cls_cE[cls] * (curl - jp);
}

template <typename T>
__global__ void __launch_bounds__(256) k_update_E(Grid<T> g, Fields<T> f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    if (i >= nx || j >= ny || k >= nz) return;
    const long long sy = nx, sz = (long long)nx * ny;
    const long long e = k * sz + j * sy + i;

    // held tangential edges on non-periodic faces
    const bool fx = !g.per[0] && i == 0, fy = !g.per[1] && j == 0, fz = !g.per[2] && k == 0;
    const bool doX = !(fy || fz), doY = !(fx || fz), doZ = !(fx || fy);

    // backward neighbour offsets (wrap on periodic axes; unused on held edges)
    const long long oim = i > 0 ? 1 : (g.per[0] ? -(long long)(nx - 1) : 0);
    const long long ojm = j > 0 ? sy : (g.per[1] ? -(long long)(ny - 1) * sy : 0);
    const long long okm = k > 0 ? sz : (g.per[2] ? -(long long)(nz - 1) * sz : 0);

    const T *Hx = f.H[0], *Hy = f.H[1], *Hz = f.H[2];
    const T hx = Hx[e], hy = Hy[e], hz = Hz[e];
    const int s0 = slab_pos(g, 0, i), s1 = slab_pos(g, 1, j), s2 = slab_pos(g, 2, k);

    if (doX) {
        const T dHz_dy = (hz - Hz[e - ojm]) * g.r[1];
        const T dHy_dz = (hy - Hy[e - okm]) * g.r[2];
        T ky = T(1), kz = T(1), py = T(0), pz = T(0);
        if (s1 >= 0) {
            ky = f.ikE[1][j];
            const long long q = psi_at(g, 1, s1, i, j, k);
            py = f.psiE[1][1][q] + (f.bE[1][j] * f.psiE[1][1][q] + f.aE[1][j] * dHz_dy); f.psiE[1][1][q] = py;
        }
        if (s2 >= 0) {
            kz = f.ikE[2][k];
            const long long q = psi_at(g, 2, s2, i, j, k);
            pz = f.psiE[2][0][q] + (f.bE[2][k] * f.psiE[2][0][q] + f.aE[2][k] * dHy_dz); f.psiE[2][0][q] = pz;
        }
        ampere(f, 0, e, ky * dHz_dy + py - kz * dHy_dz - pz);
    }
    if (doY) {
        const T dHx_dz = (hx - Hx[e - okm]) * g.r[2];
        const T dHz_dx = (hz - Hz[e - oim]) * g.r[0];
        T kz = T(1), kx = T(1), pz = T(0), px = T(0);
        if (s2 >= 0) {
            kz = f.ikE[2][k];
            const long long q = psi_at(g, 2, s2, i, j, k);
            pz = f.psiE[2][1][q] + (f.bE[2][k] * f.psiE[2][1][q] + f.aE[2][k] * dHx_dz); f.psiE[2][1][q] = pz;
        }
        if (s0 >= 0) {
            kx = f.ikE[0][i];
            const long long q = psi_at(g, 0, s0, i, j, k);
            px = f.psiE[0][0][q] + (f.bE[0][i] * f.psiE[0][0][q] + f.aE[0][i] * dHz_dx); f.psiE[0][0][q] = px;
        }
        ampere(f, 1, e, kz * dHx_dz + pz - kx * dHz_dx - px);
    }
    if (doZ) {
        const T dHy_dx = (hy - Hy[e - oim]) * g.r[0];
        const T dHx_dy = (hx - Hx[e - ojm]) * g.r[1];
        T kx = T(1), ky = T(1), px = T(0), py = T(0);
        if (s0 >= 0) {
            kx = f.ikE[0][i];
            const long long q = psi_at(g, 0, s0, i, j, k);
            px = f.psiE[0][1][q] + (f.bE[0][i] * f.psiE[0][1][q] + f.aE[0][i] * dHy_dx); f.psiE[0][1][q] = px;
        }
        if (s1 >= 0) {
            ky = f.ikE[1][j];
            const long long q = psi_at(g, 1, s1, i, j, k);
            py = f.psiE[1][0][q] + (f.bE[1][j] * f.psiE[1][0][q] + f.aE[1][j] * dHx_dy); f.psiE[1][0][q] = py;
        }
        ampere(f, 2, e, kx * dHy_dx + px - ky * dHx_dy - py);
    }
}

// The free-current term of Eq. 8, applied after the E update of the same
// step: E -= (dt/(eps0 eps_inf)) J_f on every updated edge of the tiles the
// deposit and the sources wrote this step (each listed once).  One thread per
// cell of a TILE_X x TILE_Y x TILE_Z tile; blocks stride over the list.
template <typename T>
__global__ void __launch_bounds__(TILE_X *TILE_Y *TILE_Z) k_jf_apply(Grid<T> g, Fields<T> f) {
    pdl_wait();
    pdl_release();
    const int count = *f.jf_count;
    const int i0 = threadIdx.x % TILE_X, j0 = (threadIdx.x / TILE_X) % TILE_Y, k0 = threadIdx.x / (TILE_X * TILE_Y);
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const long long t = f.jf_list[q];
        const int tx = (int)(t % g.nt[0]), ty = (int)((t / g.nt[0]) % g.nt[1]);
        const int tz = (int)(t / ((long long)g.nt[0] * g.nt[1]));
        const int i = tx * TILE_X + i0, j = ty * TILE_Y + j0, k = tz * TILE_Z + k0;
        if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) continue;
        const long long e = ((long long)k * g.n[1] + j) * g.n[0] + i;
        const bool fx = !g.per[0] && i == 0, fy = !g.per[1] && j == 0, fz = !g.per[2] && k == 0;
        const bool upd[3] = {!(fy || fz), !(fx || fz), !(fx || fy)};
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const T jf = f.Jf[c][e];
            if (upd[c] && jf != T(0)) f.E[c][e] -= f.cls_cE[f.ecls[c][e]] * jf;
        }
    }
}

// Scan of the field state for NaN or Inf (a diverged run: too large a time
// step for a material, or a non-finite value written by pic_set_field).
template <typename T>
__global__ void __launch_bounds__(256) k_nonfinite(Fields<T> f, long long n, int *err) {
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; c++) bad |= !isfinite(f.E[c][i]) || !isfinite(f.H[c][i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, DEVERR_FIELD_NONFINITE);
}

template <typename T>
void launch_nonfinite_scan(const Fields<T> &f, long long n, int *err, cudaStream_t s) {
    long long nblk = (n + 255) / 256;
    if (nblk > 8 * 152) nblk = 8 * 152;
    if (nblk < 1) nblk = 1;
    k_nonfinite<T><<<(unsigned)nblk, 256, 0, s>>>(f, n, err);
}
template void launch_nonfinite_scan<float>(const Fields<float> &, long long, int *, cudaStream_t);
template void launch_nonfinite_scan<double>(const Fields<double> &, long long, int *, cudaStream_t);

static dim3 field_grid(const int n[3], dim3 blk) {
    return dim3((n[0] + blk.x - 1) / blk.x, (n[1] + blk.y - 1) / blk.y, (n[2] + blk.z - 1) / blk.z);
}

template <typename T>
void launch_update_H(const Grid<T> &g, const Fields<T> &f, const FieldPlan *, cudaStream_t s, cudaStream_t) {
    dim3 blk(32, 4, 2);
    k_update_H<T><<<field_grid(g.n, blk), blk, 0, s>>>(g, f);
    launch_count() += 1;
}

template <typename T>
void launch_update_E(const Grid<T> &g, const Fields<T> &f, const FieldPlan *, cudaStream_t s, cudaStream_t,
                     cudaStream_t, cudaStream_t) {
    dim3 blk(32, 4, 2);
    k_update_E<T><<<field_grid(g.n, blk), blk, 0, s>>>(g, f);
    launch_count() += 1;
}

// FP32 with a plan (nx a multiple of 4): the four-cells-per-thread kernels of fields_v4.cu.
template <>
void launch_update_H<float>(const Grid<float> &g, const Fields<float> &f, const FieldPlan *plan, cudaStream_t s,
                            cudaStream_t s2) {
    dim3 blk(32, 4, 2);
    if (plan) {
        launch_v4_H(g, f, *plan, s, s2);
    } else {
        k_update_H<float><<<field_grid(g.n, blk), blk, 0, s>>>(g, f);
        launch_count() += 1;
    }
}

template <>
void launch_update_E<float>(const Grid<float> &g, const Fields<float> &f, const FieldPlan *plan, cudaStream_t s,
                            cudaStream_t s2, cudaStream_t s3, cudaStream_t s4) {
    dim3 blk(32, 4, 2);
    if (plan) {
        launch_v4_E(g, f, *plan, s, s2, s3, s4);
    } else {
        k_update_E<float><<<field_grid(g.n, blk), blk, 0, s>>>(g, f);
        launch_count() += 1;
    }
}

template <typename T>
void launch_jf_apply(const Grid<T> &g, const Fields<T> &f, int max_tiles, cudaStream_t s) {
    int nblk = max_tiles < 4 * 152 ? max_tiles : 4 * 152;
    if (nblk < 1) nblk = 1;
    launch_pdl(k_jf_apply<T>, dim3(nblk), dim3(TILE_X * TILE_Y * TILE_Z), 0, s, g, f);
    launch_count() += 1;
}

template void launch_update_H<double>(const Grid<double> &, const Fields<double> &, const FieldPlan *, cudaStream_t,
                                      cudaStream_t);
template void launch_update_E<double>(const Grid<double> &, const Fields<double> &, const FieldPlan *, cudaStream_t,
                                      cudaStream_t, cudaStream_t, cudaStream_t);

template void launch_jf_apply<float>(const Grid<float> &, const Fields<float> &, int, cudaStream_t);
template void launch_jf_apply<double>(const Grid<double> &, const Fields<double> &, int, cudaStream_t);

}  // namespace pic
