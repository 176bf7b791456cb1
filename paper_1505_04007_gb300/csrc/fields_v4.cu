// fields_v4.cu -- FP32 field updates with four consecutive x cells per thread.
//
// Every centre, row and plane access is one 16-byte load, which keeps enough
// bytes in flight to stream the grid near the HBM copy rate.  The grid is cut
// (make_field_plan) into an interior box without absorbing layers and face
// boxes over the CPML slabs, and both are cut again by z-runs into planes of
// one uniform non-metal material and planes holding metal or mixed
// materials.  Each piece gets a kernel compiled for exactly what it needs, so
// the bulk of the grid runs code with no CPML or material branches at all.
// The pieces write disjoint cells, so the split adds no traffic.  Per cell
// the arithmetic is that of the scalar kernels in fields.cu (same curl,
// increment forms, held tangential edges).
//
// Requires nx % 4 == 0 and, with CPML along x, cpml_cells % 4 == 0, so a
// four-cell group is either wholly inside an x slab or wholly outside.
#include "pic_internal.cuh"

namespace pic {

namespace {

struct F4 {
    float v[4];
};
__device__ __forceinline__ F4 ld4(const float *p) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    return F4{{q.x, q.y, q.z, q.w}};
}
__device__ __forceinline__ void st4(float *p, const F4 &a) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
__device__ __forceinline__ F4 zero4() { return F4{{0.f, 0.f, 0.f, 0.f}}; }

__device__ __forceinline__ int slab(const Grid<float> &g, int a, int x) {
    if (!g.cpml[a]) return -1;
    if (x < g.L) return x;
    if (x >= g.n[a] - g.L) return x - (g.n[a] - 2 * g.L);
    return -1;
}
__device__ __forceinline__ long long psi_idx(const Grid<float> &g, int a, int s, int i, int j, int k) {
    const long long L2 = 2 * g.L;
    if (a == 0) return ((long long)k * g.n[1] + j) * L2 + s;
    if (a == 1) return ((long long)k * L2 + s) * g.n[0] + i;
    return ((long long)s * g.n[1] + j) * g.n[0] + i;
}

// H^{n+1/2} for cells i0..i0+3 of row (j, k).
template <bool CPML>
__device__ __forceinline__ void h4(const Grid<float> &g, const Fields<float> &f, int i0, int j, int k,
                                   long long step) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long sy = nx, sz = (long long)nx * ny;
    const long long e = k * sz + j * sy + i0;

    // clear the free current the previous step deposited in this tile
    const long long t = ((long long)(k / TILE_Z) * g.nt[1] + j / TILE_Y) * g.nt[0] + i0 / TILE_X;
    if (step > 0 && f.jf_flag[t] == (int)step) {
#pragma unroll
        for (int c = 0; c < 3; c++) st4(f.Jf[c] + e, zero4());
    }

    const bool hjp = (j + 1 < ny) || g.per[1];
    const bool hkp = (k + 1 < nz) || g.per[2];
    const bool hip = (i0 + 4 < nx) || g.per[0];
    const long long ojp = (j + 1 < ny) ? sy : -(long long)(ny - 1) * sy;
    const long long okp = (k + 1 < nz) ? sz : -(long long)(nz - 1) * sz;
    const long long oip = (i0 + 4 < nx) ? 4 : -(long long)(nx - 4);

    const F4 ex = ld4(f.E[0] + e), ey = ld4(f.E[1] + e), ez = ld4(f.E[2] + e);
    const F4 ez_jp = hjp ? ld4(f.E[2] + e + ojp) : zero4();
    const F4 ex_jp = hjp ? ld4(f.E[0] + e + ojp) : zero4();
    const F4 ey_kp = hkp ? ld4(f.E[1] + e + okp) : zero4();
    const F4 ex_kp = hkp ? ld4(f.E[0] + e + okp) : zero4();
    const float ez_ip = hip ? f.E[2][e + oip] : 0.f;
    const float ey_ip = hip ? f.E[1][e + oip] : 0.f;
    F4 hx = ld4(f.H[0] + e), hy = ld4(f.H[1] + e), hz = ld4(f.H[2] + e);

    const float rx = g.r[0], ry = g.r[1], rz = g.r[2];
    float dEz_dy[4], dEy_dz[4], dEx_dz[4], dEz_dx[4], dEy_dx[4], dEx_dy[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const float ezn = m < 3 ? ez.v[m + 1] : ez_ip;
        const float eyn = m < 3 ? ey.v[m + 1] : ey_ip;
        dEz_dy[m] = (ez_jp.v[m] - ez.v[m]) * ry;
        dEy_dz[m] = (ey_kp.v[m] - ey.v[m]) * rz;
        dEx_dz[m] = (ex_kp.v[m] - ex.v[m]) * rz;
        dEz_dx[m] = (ezn - ez.v[m]) * rx;
        dEy_dx[m] = (eyn - ey.v[m]) * rx;
        dEx_dy[m] = (ex_jp.v[m] - ex.v[m]) * ry;
    }
    if (!CPML) {
#pragma unroll
        for (int m = 0; m < 4; m++) {
            hx.v[m] -= g.cH * (dEz_dy[m] - dEy_dz[m]);
            hy.v[m] -= g.cH * (dEx_dz[m] - dEz_dx[m]);
            hz.v[m] -= g.cH * (dEy_dx[m] - dEx_dy[m]);
        }
    } else {
        // Each axis adds its terms to the three curl sums in turn (its
        // profile and psi values are dead once added), which keeps the
        // register count close to the interior kernel's.
        float cx[4] = {0.f, 0.f, 0.f, 0.f}, cy[4] = {0.f, 0.f, 0.f, 0.f}, cz[4] = {0.f, 0.f, 0.f, 0.f};
        {   // x: Hy -= d/dx Ez, Hz += d/dx Ey
            const int sp = slab(g, 0, i0);
            if (sp >= 0) {
                const long long q = psi_idx(g, 0, sp, i0, j, k);
                const F4 b = ld4(f.bH[0] + i0), a = ld4(f.aH[0] + i0), ik = ld4(f.ikH[0] + i0);
                F4 p0 = ld4(f.psiH[0][0] + q), p1 = ld4(f.psiH[0][1] + q);
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    p0.v[m] += b.v[m] * p0.v[m] + a.v[m] * dEz_dx[m];
                    p1.v[m] += b.v[m] * p1.v[m] + a.v[m] * dEy_dx[m];
                    cy[m] -= ik.v[m] * dEz_dx[m] + p0.v[m];
                    cz[m] += ik.v[m] * dEy_dx[m] + p1.v[m];
                }
                st4(f.psiH[0][0] + q, p0);
                st4(f.psiH[0][1] + q, p1);
            } else {
#pragma unroll
                for (int m = 0; m < 4; m++) { cy[m] -= dEz_dx[m]; cz[m] += dEy_dx[m]; }
            }
        }
        {   // y: Hz -= d/dy Ex, Hx += d/dy Ez
            const int sp = slab(g, 1, j);
            if (sp >= 0) {
                const long long q = psi_idx(g, 1, sp, i0, j, k);
                const float b = f.bH[1][j], a = f.aH[1][j], ik = f.ikH[1][j];
                F4 p0 = ld4(f.psiH[1][0] + q), p1 = ld4(f.psiH[1][1] + q);
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    p0.v[m] += b * p0.v[m] + a * dEx_dy[m];
                    p1.v[m] += b * p1.v[m] + a * dEz_dy[m];
                    cz[m] -= ik * dEx_dy[m] + p0.v[m];
                    cx[m] += ik * dEz_dy[m] + p1.v[m];
                }
                st4(f.psiH[1][0] + q, p0);
                st4(f.psiH[1][1] + q, p1);
            } else {
#pragma unroll
                for (int m = 0; m < 4; m++) { cz[m] -= dEx_dy[m]; cx[m] += dEz_dy[m]; }
            }
        }
        {   // z: Hx -= d/dz Ey, Hy += d/dz Ex
            const int sp = slab(g, 2, k);
            if (sp >= 0) {
                const long long q = psi_idx(g, 2, sp, i0, j, k);
                const float b = f.bH[2][k], a = f.aH[2][k], ik = f.ikH[2][k];
                F4 p0 = ld4(f.psiH[2][0] + q), p1 = ld4(f.psiH[2][1] + q);
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    p0.v[m] += b * p0.v[m] + a * dEy_dz[m];
                    p1.v[m] += b * p1.v[m] + a * dEx_dz[m];
                    cx[m] -= ik * dEy_dz[m] + p0.v[m];
                    cy[m] += ik * dEx_dz[m] + p1.v[m];
                }
                st4(f.psiH[2][0] + q, p0);
                st4(f.psiH[2][1] + q, p1);
            } else {
#pragma unroll
                for (int m = 0; m < 4; m++) { cx[m] -= dEy_dz[m]; cy[m] += dEx_dz[m]; }
            }
        }
#pragma unroll
        for (int m = 0; m < 4; m++) {
            hx.v[m] -= g.cH * cx[m];
            hy.v[m] -= g.cH * cy[m];
            hz.v[m] -= g.cH * cz[m];
        }
    }
    st4(f.H[0] + e, hx);
    st4(f.H[1] + e, hy);
    st4(f.H[2] + e, hz);
}

// Eq. 6 (increment form) on the metal edges among the four, then Eq. 8
// without the free current (applied by k_jf_apply after the deposit), for
// component comp of cells e..e+3 with edge classes cl; J_p moves as one
// 16-byte access when any of the four edges is metal.
__device__ __forceinline__ void ampere4(const Fields<float> &f, int comp, uchar4 cl, long long e, F4 &E, const float curl[4],
                                        const bool doit[4]) {
    const float4 t0 = f.cls_pack[cl.x], t1 = f.cls_pack[cl.y], t2 = f.cls_pack[cl.z], t3 = f.cls_pack[cl.w];
    const float4 t[4] = {t0, t1, t2, t3};
    const bool metal = (t0.w + t1.w + t2.w + t3.w) != 0.f;
    F4 jp = zero4();
    if (metal) {
        jp = ld4(f.Jp[comp] + e);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const float j0 = jp.v[m];
            jp.v[m] = (t[m].w != 0.f && doit[m]) ? j0 + (t[m].x * j0 + t[m].y * E.v[m]) : j0;
        }
        st4(f.Jp[comp] + e, jp);
    }
#pragma unroll
    for (int m = 0; m < 4; m++)
        if (doit[m]) E.v[m] += t[m].z * (curl[m] - (t[m].w != 0.f ? jp.v[m] : 0.f));
}

// E^{n+1} (with the Drude current of Eq. 6) for cells i0..i0+3 of row (j, k).
// MAT: per-edge material classes (else every edge has the Ampere factor cEu
// of one non-metal material and carries no polarisation current).
template <bool CPML, bool MAT>
__device__ __forceinline__ void e4(const Grid<float> &g, const Fields<float> &f, int i0, int j, int k,
                                   long long step, float cEu) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long sy = nx, sz = (long long)nx * ny;
    const long long e = k * sz + j * sy + i0;

    const bool fx0 = !g.per[0] && i0 == 0;  // only cell m = 0 can sit on the x face
    const bool fy = !g.per[1] && j == 0, fz = !g.per[2] && k == 0;
    const long long ojm = j > 0 ? sy : (g.per[1] ? -(long long)(ny - 1) * sy : 0);
    const long long okm = k > 0 ? sz : (g.per[2] ? -(long long)(nz - 1) * sz : 0);
    const long long oim = i0 > 0 ? 1 : (g.per[0] ? -(long long)(nx - 1) : 0);

    (void)step;

    const F4 hx = ld4(f.H[0] + e), hy = ld4(f.H[1] + e), hz = ld4(f.H[2] + e);
    const F4 hz_jm = ld4(f.H[2] + e - ojm), hx_jm = ld4(f.H[0] + e - ojm);
    const F4 hy_km = ld4(f.H[1] + e - okm), hx_km = ld4(f.H[0] + e - okm);
    const float hz_im = f.H[2][e - oim], hy_im = f.H[1][e - oim];
    F4 ex = ld4(f.E[0] + e), ey = ld4(f.E[1] + e), ez = ld4(f.E[2] + e);
    uchar4 cl0 = make_uchar4(0, 0, 0, 0), cl1 = cl0, cl2 = cl0;
    if (MAT) {
        cl0 = *reinterpret_cast<const uchar4 *>(f.ecls[0] + e);
        cl1 = *reinterpret_cast<const uchar4 *>(f.ecls[1] + e);
        cl2 = *reinterpret_cast<const uchar4 *>(f.ecls[2] + e);
    }

    const float rx = g.r[0], ry = g.r[1], rz = g.r[2];
    float dHz_dy[4], dHy_dz[4], dHx_dz[4], dHz_dx[4], dHy_dx[4], dHx_dy[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const float hzm = m > 0 ? hz.v[m - 1] : hz_im;
        const float hym = m > 0 ? hy.v[m - 1] : hy_im;
        dHz_dy[m] = (hz.v[m] - hz_jm.v[m]) * ry;
        dHy_dz[m] = (hy.v[m] - hy_km.v[m]) * rz;
        dHx_dz[m] = (hx.v[m] - hx_km.v[m]) * rz;
        dHz_dx[m] = (hz.v[m] - hzm) * rx;
        dHy_dx[m] = (hy.v[m] - hym) * rx;
        dHx_dy[m] = (hx.v[m] - hx_jm.v[m]) * ry;
    }
    // curl sums, one axis at a time (in the absorbing slabs with psi and
    // 1/kappa); a held edge (E stays zero) leaves its psi untouched
    float cx[4], cy[4], cz[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        cx[m] = dHz_dy[m] - dHy_dz[m];
        cy[m] = dHx_dz[m] - dHz_dx[m];
        cz[m] = dHy_dx[m] - dHx_dy[m];
    }
    if (CPML) {
        {   // x: Ey -= d/dx Hz, Ez += d/dx Hy
            const int sp = slab(g, 0, i0);
            if (sp >= 0) {
                const long long q = psi_idx(g, 0, sp, i0, j, k);
                const F4 b = ld4(f.bE[0] + i0), a = ld4(f.aE[0] + i0), ik = ld4(f.ikE[0] + i0);
                F4 p0 = ld4(f.psiE[0][0] + q), p1 = ld4(f.psiE[0][1] + q);
                const float o0 = p0.v[0], o1 = p1.v[0];
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    p0.v[m] += b.v[m] * p0.v[m] + a.v[m] * dHz_dx[m];
                    p1.v[m] += b.v[m] * p1.v[m] + a.v[m] * dHy_dx[m];
                    cy[m] += (1.f - ik.v[m]) * dHz_dx[m] - p0.v[m];
                    cz[m] += (ik.v[m] - 1.f) * dHy_dx[m] + p1.v[m];
                }
                if (fx0) { p0.v[0] = o0; p1.v[0] = o1; }
                if (!fz) st4(f.psiE[0][0] + q, p0);
                if (!fy) st4(f.psiE[0][1] + q, p1);
            }
        }
        {   // y: Ez -= d/dy Hx, Ex += d/dy Hz
            const int sp = slab(g, 1, j);
            if (sp >= 0) {
                const long long q = psi_idx(g, 1, sp, i0, j, k);
                const float b = f.bE[1][j], a = f.aE[1][j], ik = f.ikE[1][j];
                F4 p0 = ld4(f.psiE[1][0] + q), p1 = ld4(f.psiE[1][1] + q);
                const float o0 = p0.v[0];
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    p0.v[m] += b * p0.v[m] + a * dHx_dy[m];
                    p1.v[m] += b * p1.v[m] + a * dHz_dy[m];
                    cz[m] += (1.f - ik) * dHx_dy[m] - p0.v[m];
                    cx[m] += (ik - 1.f) * dHz_dy[m] + p1.v[m];
                }
                if (fx0) p0.v[0] = o0;
                if (!fy) st4(f.psiE[1][0] + q, p0);
                if (!(fy || fz)) st4(f.psiE[1][1] + q, p1);
            }
        }
        {   // z: Ex -= d/dz Hy, Ey += d/dz Hx
            const int sp = slab(g, 2, k);
            if (sp >= 0) {
                const long long q = psi_idx(g, 2, sp, i0, j, k);
                const float b = f.bE[2][k], a = f.aE[2][k], ik = f.ikE[2][k];
                F4 p0 = ld4(f.psiE[2][0] + q), p1 = ld4(f.psiE[2][1] + q);
                const float o1 = p1.v[0];
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    p0.v[m] += b * p0.v[m] + a * dHy_dz[m];
                    p1.v[m] += b * p1.v[m] + a * dHx_dz[m];
                    cx[m] += (1.f - ik) * dHy_dz[m] - p0.v[m];
                    cy[m] += (ik - 1.f) * dHx_dz[m] + p1.v[m];
                }
                if (fx0) p1.v[0] = o1;
                if (!(fy || fz)) st4(f.psiE[2][0] + q, p0);
                if (!fz) st4(f.psiE[2][1] + q, p1);
            }
        }
    }
    bool doX[4], doY[4], doZ[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const bool fx = fx0 && m == 0;
        doX[m] = !(fy || fz);
        doY[m] = !(fx || fz);
        doZ[m] = !(fx || fy);
    }
    if (MAT) {
        ampere4(f, 0, cl0, e, ex, cx, doX);
        ampere4(f, 1, cl1, e, ey, cy, doY);
        ampere4(f, 2, cl2, e, ez, cz, doZ);
    } else {
#pragma unroll
        for (int m = 0; m < 4; m++) {
            if (doX[m]) ex.v[m] += cEu * cx[m];
            if (doY[m]) ey.v[m] += cEu * cy[m];
            if (doZ[m]) ez.v[m] += cEu * cz[m];
        }
    }
    st4(f.E[0] + e, ex);
    st4(f.E[1] + e, ey);
    st4(f.E[2] + e, ez);
}

// Thread -> cell group: the groups of all boxes of a list are numbered one
// after the other, so every block has work whatever the box sizes.
__device__ __forceinline__ bool list_cell(const BoxList &bl, long long q, int &bi, int &i0, int &j, int &k) {
    if (q >= bl.first[bl.n]) return false;
    bi = 0;
    while (q >= bl.first[bi + 1]) bi++;
    const Box &b = bl.b[bi];
    // 32-bit arithmetic: a plan exists only for grids of fewer than 2^31 four-cell groups
    const unsigned r = (unsigned)(q - bl.first[bi]);
    const unsigned wx = (unsigned)(b.hi[0] - b.lo[0]) / 4u, wy = (unsigned)(b.hi[1] - b.lo[1]);
    const unsigned row = r / wx, kk = row / wy;
    i0 = b.lo[0] + 4 * (int)(r - row * wx);
    j = b.lo[1] + (int)(row - kk * wy);
    k = b.lo[2] + (int)kk;
    return true;
}

#define BOX_CELL(bl)                                                                                   \
    pdl_wait();                                                                                        \
    pdl_release();                                                                                     \
    int bi, i0, j, k;                                                                                  \
    if (!list_cell((bl), blockIdx.x * (long long)blockDim.x + threadIdx.x, bi, i0, j, k)) return;      \
    const Box &b = (bl).b[bi];                                                                         \
    (void)b;

__global__ void __launch_bounds__(512) k_H4_bulk(Grid<float> g, Fields<float> f, BoxList bl) {
    BOX_CELL(bl);
    h4<false>(g, f, i0, j, k, *f.step);
}
__global__ void __launch_bounds__(256, 3) k_H4_cpml(Grid<float> g, Fields<float> f, BoxList bl) {
    BOX_CELL(bl);
    h4<true>(g, f, i0, j, k, *f.step);
}
// one non-metal material, no absorbing layer
__global__ void __launch_bounds__(512) k_E4_vac(Grid<float> g, Fields<float> f, BoxList bl) {
    BOX_CELL(bl);
    e4<false, false>(g, f, i0, j, k, *f.step, b.cE);
}
// metal or several materials, no absorbing layer (256-thread blocks: its
// register count would rise above 80 under a 512-thread bound)
__global__ void __launch_bounds__(256) k_E4_mat(Grid<float> g, Fields<float> f, BoxList bl) {
    BOX_CELL(bl);
    e4<false, true>(g, f, i0, j, k, *f.step, 0.f);
}
// one non-metal material inside the absorbing slabs
__global__ void __launch_bounds__(256, 3) k_E4_cpml_vac(Grid<float> g, Fields<float> f, BoxList bl) {
    BOX_CELL(bl);
    e4<true, false>(g, f, i0, j, k, *f.step, b.cE);
}
// metal or several materials inside the absorbing slabs
__global__ void __launch_bounds__(256) k_E4_cpml_mat(Grid<float> g, Fields<float> f, BoxList bl) {
    BOX_CELL(bl);
    e4<true, true>(g, f, i0, j, k, *f.step, 0.f);
}

long long groups(const Box &b) {
    return (long long)((b.hi[0] - b.lo[0]) / 4) * (b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]);
}

template <typename K>
void launch_list(K kernel, const Grid<float> &g, const Fields<float> &f, const BoxList &bl, cudaStream_t s,
                 int blk = 256) {
    const long long total = bl.first[bl.n];
    if (total > 0) {
        launch_pdl(kernel, dim3((unsigned)((total + blk - 1) / blk)), dim3(blk), 0, s, g, f, bl);
        launch_count() += 1;
    }
}

bool add_box(BoxList &bl, int x0, int x1, int y0, int y1, int z0, int z1, float cE) {
    if (!(x1 > x0 && y1 > y0 && z1 > z0)) return true;
    if (bl.n >= MAX_BOXES) return false;
    bl.b[bl.n] = Box{{x0, y0, z0}, {x1, y1, z1}, cE};
    bl.first[bl.n + 1] = bl.first[bl.n] + groups(bl.b[bl.n]);
    bl.n++;
    return true;
}

// Cut a box by z-runs of plane class into the vacuum list (one non-metal
// class per run) and the material list.
bool split_by_planes(const int lo[3], const int hi[3], const uint8_t *plane_cls, const float *cls_cE, BoxList &vac,
                     BoxList &mat) {
    int k = lo[2];
    while (k < hi[2]) {
        int k1 = k + 1;
        while (k1 < hi[2] && plane_cls[k1] == plane_cls[k]) k1++;
        const bool uniform = plane_cls[k] != 255;
        if (!add_box(uniform ? vac : mat, lo[0], hi[0], lo[1], hi[1], k, k1, uniform ? cls_cE[plane_cls[k]] : 0.f))
            return false;
        k = k1;
    }
    return true;
}

}  // namespace

bool make_field_plan(const Grid<float> &g, const uint8_t *plane_cls, const float *cls_cE, FieldPlan &p) {
    p = FieldPlan{};
    if (g.n[0] % 4 != 0 || (g.cpml[0] && g.L % 4 != 0)) return false;
    if ((long long)g.n[0] * g.n[1] * g.n[2] / 4 >= (1LL << 31)) return false;  // list_cell indexes in 32 bits
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = g.cpml[a] ? g.L : 0;
        hi[a] = g.cpml[a] ? g.n[a] - g.L : g.n[a];
    }
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    // interior box and the face boxes around it (a partition of the grid)
    add_box(p.bulk, lo[0], hi[0], lo[1], hi[1], lo[2], hi[2], 0.f);
    const int faces[6][6] = {{0, nx, 0, ny, 0, lo[2]},
                             {0, nx, 0, ny, hi[2], nz},
                             {0, nx, 0, lo[1], lo[2], hi[2]},
                             {0, nx, hi[1], ny, lo[2], hi[2]},
                             {0, lo[0], lo[1], hi[1], lo[2], hi[2]},
                             {hi[0], nx, lo[1], hi[1], lo[2], hi[2]}};
    for (auto &fb : faces) add_box(p.faces, fb[0], fb[1], fb[2], fb[3], fb[4], fb[5], 0.f);
    // E: the same partition, cut by plane material
    if (!split_by_planes(lo, hi, plane_cls, cls_cE, p.vac, p.mat)) return false;
    for (auto &fb : faces) {
        const int flo[3] = {fb[0], fb[2], fb[4]}, fhi[3] = {fb[1], fb[3], fb[5]};
        if (flo[0] >= fhi[0] || flo[1] >= fhi[1] || flo[2] >= fhi[2]) continue;
        if (!split_by_planes(flo, fhi, plane_cls, cls_cE, p.fvac, p.fmat)) return false;
    }
    return true;
}

void launch_v4_H(const Grid<float> &g, const Fields<float> &f, const FieldPlan &plan, cudaStream_t s, cudaStream_t s2) {
    launch_list(k_H4_cpml, g, f, plan.faces, s2);
    launch_list(k_H4_bulk, g, f, plan.bulk, s, plan.block);
}

void launch_v4_E(const Grid<float> &g, const Fields<float> &f, const FieldPlan &plan, cudaStream_t s, cudaStream_t s2,
                 cudaStream_t s3, cudaStream_t s4) {
    launch_list(k_E4_cpml_vac, g, f, plan.fvac, s2);
    launch_list(k_E4_cpml_mat, g, f, plan.fmat, s4);
    launch_list(k_E4_vac, g, f, plan.vac, s, plan.block);
    launch_list(k_E4_mat, g, f, plan.mat, s3);
}

}  // namespace pic
