// fields_fused.cu -- the FP32 field updates of one step as a single pass over
// the grid: E^{n+1} (Eq. 6 then Eq. 8, without the free current) and then
// H^{n+3/2} (the vacuum Yee update of the next step), with their CPML terms.
//
// Why one pass: the two updates of a step, run one after the other, read E
// and H twice and write each once (72 bytes per FP32 cell); the fused pass
// reads each once and writes each once (48 bytes).  H^{n+3/2} needs E^{n+1}
// of its own cell and of the cells at +x, +y, +z, so a block marches up a
// column of planes: it computes E^{n+1} of plane z, then H^{n+3/2} of plane
// z-1, keeping the planes it needs in shared memory.
//
// Layout of a work item: a tile of TX x TY cells (x, y) over a run of `chunk`
// planes.  A thread owns four consecutive x cells of one row (TX/4 threads
// per row).  H^{n+3/2} at the tile's last column and row needs E^{n+1} one
// cell beyond the tile, which belongs to the neighbouring tile: the last
// thread of each row also computes that row's cell at x0+TX, and one more
// row of threads computes the row y0+TY; the chunk's last E plane is
// likewise computed by both chunks that need it.  Recomputed values are
// used, never stored.  Because a neighbour may already have written its
// cells of the step, the pass reads the state at step n from one copy of
// the arrays (X) and writes step n+1 to another (Y).
//
// Tiles come in four kinds, each a kernel of its own (template K): tiles
// whose cells, halo row and halo column stay out of the x and y absorbing
// slabs (K = 0; z slabs are handled per plane), tiles that meet a y slab
// only (K = 1), an x slab only (K = 2), or both (K = 3).  The slab kinds
// stage the slab's CPML memory with E and H; they trade the third E^{n+1}
// plane and the shared class table for that staging, so that the x-only and
// y-only kinds still fit three blocks on an SM.
//
// Staging: one thread streams the planes of E^n and H^{n+1/2} into a ring of
// STAGES shared-memory slots with bulk tensor copies (cp.async.bulk.tensor,
// one copy per field and plane, the three components at once), signalled
// by mbarriers; every wait is bounded (on timeout the block records
// DEVERR_WAIT, waits a bounded time for its copies in flight and returns).
// The E^{n+1} planes go through a ring of plain shared-memory planes (three
// in the inner kind; two, with a second barrier per plane, in the slab kinds).
// A joint pass (k_fused_joint) runs the items of several simulations in one
// launch per kind, with each instance's arguments and maps from a table.
//
// What is not staged by tensor copies: per-plane and per-column/row tables
// (material factor, z-slab index and profiles, x- and y-slab profiles, the
// class table) go to shared memory once per item; the per-cell operands of
// material planes (edge classes, Drude current) and of z-slab planes (CPML
// memory) are loaded from global memory at the top of the plane's iteration,
// the halo cell's too (a load chained behind a class lookup stalled whole
// warps), and are brought into L2 two planes ahead (prefetch.global.L2).
//
// Free current: Eq. 8's J_f term is left out of the pass (the pass does not
// wait for the push, and in a batch runs beside it).  k_jf_fix adds it
// afterwards on the tiles the deposit wrote: dE = -dt/(eps0 eps_inf) J_f on
// those edges, and the change of H^{n+3/2} (and of its CPML memory) that dE
// causes through the H update, which is linear in E.
#include <cuda.h>

#include <mutex>
#include <type_traits>

#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int TX = FUSED_TX, TY = FUSED_TY;
constexpr int GX = 4, TPR = TX / GX;     // four x cells per thread, threads per tile row
constexpr int NT = TPR * (TY + 1);       // the tile's rows and the halo row beyond it
constexpr int STAGES = 3;
constexpr int EW = TX + 4, EH = TY + 1;  // E^n box: x0..x0+TX+3, y0..y0+TY
constexpr int HW = TX + 8, HH = TY + 2;  // H box: x0-4..x0+TX+3, y0-1..y0+TY
constexpr int EBOX_B = 3 * EH * EW * 4, HBOX_B = 3 * HH * HW * 4;  // bytes a tensor copy writes
constexpr int EBOX = (3 * EH * EW + 31) / 32 * 32;                  // floats, slots 128-byte aligned
constexpr int HBOX = (3 * HH * HW + 31) / 32 * 32;
constexpr int XW = TX + 4;               // E^{n+1} plane row: x0..x0+TX+3 (column TX: the halo cell)
constexpr int NBOX = 3 * EH * XW;
static_assert(TX % 32 == 0 && NT % 32 == 0, "whole warps");

constexpr int MAX_CHUNK = 64;
// CPML memory of the x and y slabs, staged with E and H for the tiles that
// meet those slabs.  A tile meets the slab of one face only (the grid checks
// guarantee it), so a copy takes that face's L slab columns or rows: x slabs
// [comp][row y0..y0+TY][L columns], y slabs [comp][up to FUSED_MAX_L slab
// rows][x0..x0+TX+3].
constexpr int PXW = FUSED_MAX_L, PYH = FUSED_MAX_L;
constexpr int PXBOX = 2 * EH * PXW, PYBOX = 2 * PYH * EW;  // floats (multiples of 32)
static_assert(PXBOX % 32 == 0 && PYBOX % 32 == 0, "128-byte aligned slots");

template <int K, bool J>
struct __align__(128) Smem {
    static constexpr bool XS = (K & 2) != 0, YS = (K & 1) != 0;
    static constexpr int NEN = K ? 2 : 3;  // E^{n+1} planes in the ring
    float e[STAGES][EBOX];
    float h[STAGES][HBOX];
    float pex[XS ? STAGES : 1][XS ? PXBOX : 32], phx[XS ? STAGES : 1][XS ? PXBOX : 32];  // psi_E, psi_H, x slab
    float pey[YS ? STAGES : 1][YS ? PYBOX : 32], phy[YS ? STAGES : 1][YS ? PYBOX : 32];  // ... y slab
    float en[NEN][NBOX];
    float4 cls[K ? 1 : 256];    // per edge class: kJ-1, bJ, cE, metal (the slab kinds read it from global)
    float pcE[MAX_CHUNK + 2];   // per plane of the item
    int pzs[MAX_CHUNK + 2];
    float pzp[6][MAX_CHUNK + 2];  // ... its z-slab profiles (b-1, a, 1/kappa of E, then of H; 0 outside)
    alignas(16) float prx[XS ? 6 : 1][XS ? XW : 4];  // x-slab profiles of columns x0..x0+TX+3 (same order)
    float pry[YS ? 6 : 1][YS ? EH : 1];              // y-slab profiles of rows y0..y0+TY
    unsigned long long bar[STAGES];
    int abort_flag;
    alignas(16) typename std::conditional<J, FusedArgs, int>::type args;  // a joint pass: the item's instance (copied in 16-byte pieces)
};
template <int K, bool J>
constexpr size_t smem_bytes() { return sizeof(Smem<K, J>) + 128; }  // + alignment slack
static_assert(3 * (smem_bytes<0, true>() + 1024) <= 233472 && 3 * (smem_bytes<1, true>() + 1024) <= 233472 &&
                  3 * (smem_bytes<2, true>() + 1024) <= 233472,
              "three blocks of the inner, y-slab and x-slab kinds on one SM");

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// The block's shared memory as Smem<K, J>, 128-byte aligned by pointer
// arithmetic on the dynamic array, so that accesses through it stay
// shared-memory accesses.
template <int K, bool J>
__device__ __forceinline__ Smem<K, J> &smem_of() {
    extern __shared__ __align__(128) unsigned char raw[];
    return *reinterpret_cast<Smem<K, J> *>(raw + ((128u - (smem_u32(raw) & 127u)) & 127u));
}

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of parity `parity` to complete; false after ~0.2 s.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(b, parity))
        if (global_ns() - t0 > 200000000ull) return false;
    return true;
}
// Box of a 4-D tensor map ([3][nz][ny][nx] floats) at (x, y, z, component 0).
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *m, int x, int y, int z, unsigned long long *b) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)m), "r"(x), "r"(y), "r"(z), "r"(0), "r"(smem_u32(b))
        : "memory");
}

// Bring the line holding p into L2 (no register is held for it).
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"((unsigned long long)__cvta_generic_to_global(p)));
}

__device__ __forceinline__ int slab_of(const Grid<float> &g, int a, int x) {
    if (!g.cpml[a]) return -1;
    if (x < g.L) return x;
    if (x >= g.n[a] - g.L) return x - (g.n[a] - 2 * g.L);
    return -1;
}

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
__device__ __forceinline__ V4 zero4() { return V4{{0.f, 0.f, 0.f, 0.f}}; }

// CPML curl terms of four cells: psi (p, read from X) advances as
// psi' = psi + ((b-1) psi + a d) and the term becomes (1/kappa) d + psi';
// cells whose E edge is held keep psi (and their term is not used).  The
// new psi goes to Y at q when `wr`.  Profiles per cell (x slabs) or one for
// the four (y, z slabs).
__device__ __forceinline__ void cterm4(float t[4], const V4 &p, float *pout, unsigned q, const V4 &bm, const V4 &aa,
                                       const V4 &ik, const float d[4], const bool up[4], bool wr) {
    V4 o = p;
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const float pn = p.v[m] + (bm.v[m] * p.v[m] + aa.v[m] * d[m]);
        if (up[m]) {
            o.v[m] = pn;
            t[m] = ik.v[m] * d[m] + pn;
        }
    }
    if (wr) st4(pout + q, o);
}
__device__ __forceinline__ V4 splat(float x) { return V4{{x, x, x, x}}; }

// One work item of kind K: the tile `packed` over plane chunk `chk` of the
// instance with arguments a and tensor maps tm (E, H, psi_E x, psi_H x,
// psi_E y, psi_H y).  J: a joint pass (a lives in shared memory).
template <int K, bool J>
__device__ __forceinline__ void fused_item(const FusedArgs &a, const CUtensorMap *tm, int packed, int chk) {
    constexpr bool XS = Smem<K, J>::XS, YS = Smem<K, J>::YS, SLAB = K != 0;
    constexpr int NEN = Smem<K, J>::NEN;
    Smem<K, J> &S = smem_of<K, J>();
    const Grid<float> &g = a.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], L = g.L, L2 = 2 * g.L;
    const int x0 = (packed & 0xffff) * TX, y0 = (packed >> 16) * TY;
    const int kz0 = chk * a.chunk, kz1 = min(nz, kz0 + a.chunk);
    const int lj = threadIdx.x / TPR, gx = threadIdx.x % TPR;  // row (TY: the halo row) and x group
    const int li = GX * gx;
    const bool owner = lj < TY;
    const bool xh = owner && gx == TPR - 1;  // also E of the halo cell x0+TX of this row
    const int gi = x0 + li, gj = y0 + lj, gih = x0 + TX;
    const bool inside = gi < nx && gj < ny;   // nx % 4 == 0: the group is inside or outside as a whole
    const bool inh = xh && gih < nx && gj < ny;
    const unsigned sz = (unsigned)nx * (unsigned)ny;  // cell offsets fit 32 bits on this path
    const unsigned cxy = (unsigned)gj * (unsigned)nx + (unsigned)gi;
    // slab index of the group along x and y, and of the halo cell along x (-1: none)
    int sx = -1, syb = -1, sxh = -1;
    if (XS && inside) sx = slab_of(g, 0, gi);  // L % 4 == 0: the group is in an x slab as a whole
    if (YS && inside) syb = slab_of(g, 1, gj);
    if (XS && inh) sxh = slab_of(g, 0, gih);
    const float rx = g.r[0], ry = g.r[1], rz = g.r[2], cH = g.cH;
    // held tangential E on the low faces (all axes non-periodic here): Ex at
    // j = 0 or k = 0, Ey at i = 0 or k = 0, Ez at i = 0 or j = 0
    const bool fy = gj == 0, fx0 = gi == 0;
    const int p0 = kz0 - 1, np = kz1 - p0 + 1;  // planes kz0-1 .. kz1
    // the staged slab memory of the one face this tile meets: x slab columns
    // from compact column xs0, y slab rows from compact row ys0
    const int xs0 = x0 < L ? 0 : L;
    const int ys0 = y0 < L ? y0 : max(y0, ny - L) - (ny - L2);
    const int pyh = min(PYH, L2);                             // rows of a y-slab copy
    const int pxc = EH * L, pyc = pyh * EW;                   // component strides of the copies
    const int pxo = lj * L + (sx - xs0), pyo = (syb - ys0) * EW + li;

    // bytes one stage receives: the E and H boxes, and per staged slab two
    // copies (psi_E, psi_H) of two components each
    const unsigned xbox = 2u * EH * (unsigned)L * 4u, ybox = 2u * (unsigned)pyh * EW * 4u;
    const unsigned stage_bytes = EBOX_B + HBOX_B + (XS ? 2u * xbox : 0u) + (YS ? 2u * ybox : 0u);
    // plane p0+q into slot s: E^n and H^{n+1/2} of plane z; psi_E of plane
    // z and psi_H of plane z-1 of the slab this tile meets
    auto issue = [&](int qq, int slot) {
        const int z = p0 + qq;
        mbar_expect(&S.bar[slot], stage_bytes);
        tma_load(S.e[slot], &tm[0], x0, y0, z, &S.bar[slot]);
        tma_load(S.h[slot], &tm[1], x0 - 4, y0 - 1, z, &S.bar[slot]);
        if constexpr (XS) {
            tma_load(S.pex[slot], &tm[2], xs0, y0, z, &S.bar[slot]);
            tma_load(S.phx[slot], &tm[3], xs0, y0, z - 1, &S.bar[slot]);
        }
        if constexpr (YS) {
            tma_load(S.pey[slot], &tm[4], x0, ys0, z, &S.bar[slot]);
            tma_load(S.phy[slot], &tm[5], x0, ys0, z - 1, &S.bar[slot]);
        }
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) mbar_init(&S.bar[s], 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // the first planes are on their way while the tables below load
        for (int q = 0; q < STAGES && q < np; q++) issue(q, q);
    }
    // Tables of the item in shared memory: per plane the Ampere factor of its
    // one non-metal material (-1: per-edge classes), its z-slab index (-1:
    // none) and z-slab profiles; the class table; the x- and y-slab profiles
    // of the tile.  Every value is loaded before any is stored (a store to
    // shared memory could otherwise order the loads of a joint pass's
    // arguments, which live there too, one after another).
    static_assert(MAX_CHUNK + 2 <= NT && 6 * XW <= 2 * NT && 6 * EH <= NT, "one or two table entries per thread");
    {
        const int t = threadIdx.x;
        const int z = p0 + t;
        const bool pl = t < np && z >= 0 && z < nz;
        const int sz2 = pl ? slab_of(g, 2, z) : -1;
        const bool zs = sz2 >= 0;
        const float cE = pl ? a.plane_cE[z] : 0.f;
        float pz[6];
        pz[0] = zs ? a.bE[2][z] : 0.f;
        pz[1] = zs ? a.aE[2][z] : 0.f;
        pz[2] = zs ? a.ikE[2][z] : 0.f;
        pz[3] = zs ? a.bH[2][z] : 0.f;
        pz[4] = zs ? a.aH[2][z] : 0.f;
        pz[5] = zs ? a.ikH[2][z] : 0.f;
        float4 c0 = {}, c1 = {};
        if constexpr (K == 0) {
            c0 = a.cls_pack[t];
            c1 = a.cls_pack[t + NT];
        }
        // profile r of axis ax at i: b-1, a, 1/kappa of E, then of H
        auto prof = [&](int ax, int r, int i) -> float {
            switch (r) {
                case 0: return a.bE[ax][i];
                case 1: return a.aE[ax][i];
                case 2: return a.ikE[ax][i];
                case 3: return a.bH[ax][i];
                case 4: return a.aH[ax][i];
                default: return a.ikH[ax][i];
            }
        };
        float px0 = 0.f, px1 = 0.f, py = 0.f;
        const int u1 = t + NT;
        if constexpr (XS) {
            if (x0 + t % XW < nx) px0 = prof(0, t / XW, x0 + t % XW);
            if (u1 < 6 * XW && x0 + u1 % XW < nx) px1 = prof(0, u1 / XW, x0 + u1 % XW);
        }
        if constexpr (YS)
            if (t < 6 * EH && y0 + t % EH < ny) py = prof(1, t / EH, y0 + t % EH);
        if (t < np) {
            S.pcE[t] = cE;
            S.pzs[t] = sz2;
#pragma unroll
            for (int r = 0; r < 6; r++) S.pzp[r][t] = pz[r];
        }
        if constexpr (K == 0) {
            S.cls[t] = c0;
            S.cls[t + NT] = c1;
        }
        if constexpr (XS) {
            S.prx[t / XW][t % XW] = px0;
            if (u1 < 6 * XW) S.prx[u1 / XW][u1 % XW] = px1;
        }
        if constexpr (YS)
            if (t < 6 * EH) S.pry[t / EH][t % EH] = py;
    }
    __syncthreads();
    auto cls_at = [&](unsigned k) -> float4 {
        if constexpr (K == 0) return S.cls[k];
        else return __ldg(a.cls_pack + k);
    };

    constexpr int HC = HH * HW, EC = EH * EW, NC = EH * XW;  // component strides in the boxes
    const int eo = lj * EW + li;               // this group in the E box
    const int ho = (lj + 1) * HW + (li + 4);   // ... in the H box
    const int no = lj * XW + li;               // ... in an E^{n+1} plane
    const int hoh = (lj + 1) * HW + (TX + 4);  // the halo cell in the H box
    V4 hb[3] = {zero4(), zero4(), zero4()};    // H^{n+1/2} of this group, plane z-1
    V4 ec[3] = {zero4(), zero4(), zero4()};    // E^{n+1} of this group, plane z-1
    float hbh_x = 0.f;                         // Hx of the halo cell, plane z-1
    bool ok = true;
    int q = 0;
    for (; q < np; q++) {
        const int s = q % STAGES, z = p0 + q, kh = z - 1;
        const bool doE = inside && z >= kz0 && z < nz;
        const bool doEh = inh && z >= kz0 && z < nz;
        const bool doH = owner && inside && kh >= kz0 && kh < kz1;
        const float cEu = S.pcE[q];
        const bool mat = cEu < 0.f;
        const int szb = S.pzs[q], szh = q > 0 ? S.pzs[q - 1] : -1;
        const unsigned cz = (unsigned)z * sz + cxy, chh = cz - sz;  // this group at planes z and z-1
        // ---- global loads of this iteration, issued before the wait for the
        // staged plane: z-slab CPML memory of both updates, the Drude current
        // and the edge classes of a material plane
        V4 pEz[2], pHz[2];
        unsigned qEx = 0, qEy = 0, qEz = 0, qHx = 0, qHy = 0, qHz = 0;
        if (doE) {
            if (XS && sx >= 0) qEx = ((unsigned)z * ny + gj) * L2 + sx;
            if (YS && syb >= 0) qEy = ((unsigned)z * L2 + syb) * nx + gi;
            if (szb >= 0) {
                qEz = (unsigned)szb * sz + cxy;
                pEz[0] = ld4(a.psiEi[2][0] + qEz);
                pEz[1] = ld4(a.psiEi[2][1] + qEz);
            }
        }
        if (doH) {
            if (XS && sx >= 0) qHx = ((unsigned)kh * ny + gj) * L2 + sx;
            if (YS && syb >= 0) qHy = ((unsigned)kh * L2 + syb) * nx + gi;
            if (szh >= 0) {
                qHz = (unsigned)szh * sz + cxy;
                pHz[0] = ld4(a.psiHi[2][0] + qHz);
                pHz[1] = ld4(a.psiHi[2][1] + qHz);
            }
        }
        uchar4 cl[3];
        V4 j0[3];
        if (doE && mat) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                cl[c] = *reinterpret_cast<const uchar4 *>(a.ecls[c] + cz);
                j0[c] = ld4(a.Jpi[c] + cz);
            }
        }
        // the halo cell's classes and Drude current (Ey, Ez) and z-slab memory
        // (Ey's d/dz Hx)
        unsigned char clh[2] = {0, 0};
        float jh[2] = {0.f, 0.f}, pzh = 0.f;
        if (doEh && mat) {
            const unsigned czh = cz + (unsigned)(gih - gi);
            clh[0] = a.ecls[1][czh];
            clh[1] = a.ecls[2][czh];
            jh[0] = a.Jpi[1][czh];
            jh[1] = a.Jpi[2][czh];
        }
        if (doEh && szb >= 0) pzh = a.psiEi[2][1][(unsigned)szb * sz + cxy + (unsigned)(gih - gi)];
        // ---- the same global operands of plane z+2 (E) and z+1 (H) into L2, so
        // that their loads two iterations on do not wait on DRAM: a material or
        // z-slab plane is otherwise several times slower than a vacuum one
        if (q + 2 < np && z + 2 < nz) {
            const unsigned c2 = cz + 2 * sz;
            if (S.pcE[q + 2] < 0.f) {
                if (inside) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        prefetch_l2(a.Jpi[c] + c2);
                        prefetch_l2(a.ecls[c] + c2);
                    }
                }
                if (inh) {
                    const unsigned c2h = c2 + (unsigned)(gih - gi);
                    prefetch_l2(a.Jpi[1] + c2h);
                    prefetch_l2(a.Jpi[2] + c2h);
                    prefetch_l2(a.ecls[1] + c2h);
                    prefetch_l2(a.ecls[2] + c2h);
                }
            }
            const int s2 = S.pzs[q + 2], s2h = S.pzs[q + 1];
            if (inside && s2 >= 0) {
                prefetch_l2(a.psiEi[2][0] + (unsigned)s2 * sz + cxy);
                prefetch_l2(a.psiEi[2][1] + (unsigned)s2 * sz + cxy);
            }
            if (owner && inside && s2h >= 0) {
                prefetch_l2(a.psiHi[2][0] + (unsigned)s2h * sz + cxy);
                prefetch_l2(a.psiHi[2][1] + (unsigned)s2h * sz + cxy);
            }
        }
        if (!mbar_wait(&S.bar[s], (q / STAGES) & 1)) ok = false;
        if constexpr (SLAB) {
            // every thread is done with iteration q-1: its E^{n+1} plane and
            // its staging slot are free again
            __syncthreads();
            if (threadIdx.x == 0 && q >= 1 && q - 1 + STAGES < np) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(q - 1 + STAGES, (q - 1) % STAGES);
            }
        }
        const float *e = S.e[s], *h = S.h[s];
        float *enb = S.en[q % NEN];
        V4 hc[3] = {ld4(h + ho), ld4(h + HC + ho), ld4(h + 2 * HC + ho)};
        const float hch_x = xh ? h[hoh] : 0.f;
        V4 en[3] = {zero4(), zero4(), zero4()};
        if (doE) {
            // ---- E^{n+1} of the group at plane z (Eq. 6, Eq. 8 without J_f)
            const bool wr = owner && z < kz1;  // this block owns the plane's state
            const V4 hz_jm = ld4(h + 2 * HC + ho - HW), hx_jm = ld4(h + ho - HW);
            const float hz_im = h[2 * HC + ho - 1], hy_im = h[HC + ho - 1];
            float t[6][4];  // curl terms: Ex (1,2), Ey (3,4), Ez (5,6)
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const float hzm = m ? hc[2].v[m - 1] : hz_im, hym = m ? hc[1].v[m - 1] : hy_im;
                t[0][m] = (hc[2].v[m] - hz_jm.v[m]) * ry;  // dHz/dy
                t[1][m] = (hc[1].v[m] - hb[1].v[m]) * rz;  // dHy/dz
                t[2][m] = (hc[0].v[m] - hb[0].v[m]) * rz;  // dHx/dz
                t[3][m] = (hc[2].v[m] - hzm) * rx;         // dHz/dx
                t[4][m] = (hc[1].v[m] - hym) * rx;         // dHy/dx
                t[5][m] = (hc[0].v[m] - hx_jm.v[m]) * ry;  // dHx/dy
            }
            const bool uxx = !(fy || z == 0);
            bool ux[4], uy[4], uz[4];
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const bool f0 = fx0 && m == 0;
                ux[m] = uxx;
                uy[m] = !(f0 || z == 0);
                uz[m] = !(f0 || fy);
            }
            if (XS && sx >= 0) {  // x slab: Ey's d/dx Hz, Ez's d/dx Hy (profiles per cell)
                const V4 bm = ld4(&S.prx[0][li]), aa = ld4(&S.prx[1][li]), ik = ld4(&S.prx[2][li]);
                float d3[4], d4[4];
#pragma unroll
                for (int m = 0; m < 4; m++) { d3[m] = t[3][m]; d4[m] = t[4][m]; }
                cterm4(t[3], ld4(S.pex[s] + pxo), a.psiEo[0][0], qEx, bm, aa, ik, d3, uy, wr);
                cterm4(t[4], ld4(S.pex[s] + pxc + pxo), a.psiEo[0][1], qEx, bm, aa, ik, d4, uz, wr);
            }
            if (YS && syb >= 0) {  // y slab: Ez's d/dy Hx, Ex's d/dy Hz
                const V4 bm = splat(S.pry[0][lj]), aa = splat(S.pry[1][lj]), ik = splat(S.pry[2][lj]);
                float d5[4], d0[4];
#pragma unroll
                for (int m = 0; m < 4; m++) { d5[m] = t[5][m]; d0[m] = t[0][m]; }
                cterm4(t[5], ld4(S.pey[s] + pyo), a.psiEo[1][0], qEy, bm, aa, ik, d5, uz, wr);
                cterm4(t[0], ld4(S.pey[s] + pyc + pyo), a.psiEo[1][1], qEy, bm, aa, ik, d0, ux, wr);
            }
            if (szb >= 0) {  // z slab: Ex's d/dz Hy, Ey's d/dz Hx
                const V4 bm = splat(S.pzp[0][q]), aa = splat(S.pzp[1][q]), ik = splat(S.pzp[2][q]);
                float d1[4], d2[4];
#pragma unroll
                for (int m = 0; m < 4; m++) { d1[m] = t[1][m]; d2[m] = t[2][m]; }
                cterm4(t[1], pEz[0], a.psiEo[2][0], qEz, bm, aa, ik, d1, ux, wr);
                cterm4(t[2], pEz[1], a.psiEo[2][1], qEz, bm, aa, ik, d2, uy, wr);
            }
            en[0] = ld4(e + eo);
            en[1] = ld4(e + EC + eo);
            en[2] = ld4(e + 2 * EC + eo);
            if (!mat) {  // one non-metal material on the whole plane
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    if (ux[m]) en[0].v[m] += cEu * (t[0][m] - t[1][m]);
                    if (uy[m]) en[1].v[m] += cEu * (t[2][m] - t[3][m]);
                    if (uz[m]) en[2].v[m] += cEu * (t[4][m] - t[5][m]);
                }
            } else {  // per-edge classes: Eq. 6 on metal edges, then Eq. 8
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const unsigned char k4[4] = {cl[c].x, cl[c].y, cl[c].z, cl[c].w};
                    V4 jn = j0[c];
                    bool metal = false;
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const float4 tc = cls_at(k4[m]);
                        const bool up = c == 0 ? ux[m] : (c == 1 ? uy[m] : uz[m]);
                        const float curl = t[2 * c][m] - t[2 * c + 1][m];
                        float jp = 0.f;
                        if (tc.w != 0.f) {
                            metal = true;
                            jp = up ? j0[c].v[m] + (tc.x * j0[c].v[m] + tc.y * en[c].v[m]) : j0[c].v[m];
                            jn.v[m] = jp;
                        }
                        if (up) en[c].v[m] += tc.z * (curl - jp);
                    }
                    if (wr && metal) st4(a.Jpo[c] + cz, jn);
                }
            }
        }
        if (doEh) {
            // ---- Ey, Ez of the halo cell x0+TX (one cell, the same updates)
            const float hzh = h[2 * HC + hoh], hyh = h[HC + hoh], hxh = h[hoh];
            const float hx_jmh = h[hoh - HW];
            float dHx_dz = (hxh - hbh_x) * rz, dHz_dx = (hzh - hc[2].v[3]) * rx;
            float dHy_dx = (hyh - hc[1].v[3]) * rx, dHx_dy = (hxh - hx_jmh) * ry;
            float ty1 = dHx_dz, ty2 = dHz_dx, tz1 = dHy_dx, tz2 = dHx_dy;
            const bool uyh = z != 0, uzh = !fy;
            if (XS && sxh >= 0) {
                const int ox = lj * L + (sxh - xs0);
                const float bm = S.prx[0][TX], aa = S.prx[1][TX], ik = S.prx[2][TX];
                if (uyh) { const float p = S.pex[s][ox]; ty2 = ik * dHz_dx + (p + (bm * p + aa * dHz_dx)); }
                if (uzh) { const float p = S.pex[s][pxc + ox]; tz1 = ik * dHy_dx + (p + (bm * p + aa * dHy_dx)); }
            }
            if (YS && syb >= 0 && uzh) {
                const float bm = S.pry[0][lj], aa = S.pry[1][lj], ik = S.pry[2][lj];
                const float p = S.pey[s][pyo - li + TX];
                tz2 = ik * dHx_dy + (p + (bm * p + aa * dHx_dy));
            }
            if (szb >= 0 && uyh) {
                const float bm = S.pzp[0][q], aa = S.pzp[1][q], ik = S.pzp[2][q];
                ty1 = ik * dHx_dz + (pzh + (bm * pzh + aa * dHx_dz));
            }
            float eyh = e[EC + lj * EW + TX], ezh = e[2 * EC + lj * EW + TX];
            if (!mat) {
                if (uyh) eyh += cEu * (ty1 - ty2);
                if (uzh) ezh += cEu * (tz1 - tz2);
            } else {
                const float4 ty = cls_at(clh[0]), tz = cls_at(clh[1]);
                if (uyh) {
                    float jp = 0.f;
                    if (ty.w != 0.f) jp = jh[0] + (ty.x * jh[0] + ty.y * eyh);
                    eyh += ty.z * ((ty1 - ty2) - jp);
                }
                if (uzh) {
                    float jp = 0.f;
                    if (tz.w != 0.f) jp = jh[1] + (tz.x * jh[1] + tz.y * ezh);
                    ezh += tz.z * ((tz1 - tz2) - jp);
                }
            }
            enb[NC + lj * XW + TX] = eyh;
            enb[2 * NC + lj * XW + TX] = ezh;
        } else if (xh && z >= kz0) {
            enb[NC + lj * XW + TX] = 0.f;  // beyond the high x face E reads as zero
            enb[2 * NC + lj * XW + TX] = 0.f;
        }
        if (z >= kz0) {
            st4(enb + no, en[0]);
            st4(enb + NC + no, en[1]);
            st4(enb + 2 * NC + no, en[2]);
        }
        if (!ok) S.abort_flag = 1;
        __syncthreads();
        if (S.abort_flag) break;
        if constexpr (!SLAB) {
            if (threadIdx.x == 0 && q + STAGES < np) {  // the slot read above is free again
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(q + STAGES, s);
            }
        }
        // ---- H^{n+3/2} of the group at plane kh = z-1 from E^{n+1} of planes kh and kh+1
        if (doH) {
            const float *bp = S.en[(q + NEN - 1) % NEN];  // plane kh
            const float ez_ip = bp[2 * NC + no + 4], ey_ip = bp[NC + no + 4];
            const V4 ez_jp = ld4(bp + 2 * NC + no + XW), ex_jp = ld4(bp + no + XW);
            V4 e1[3] = {en[0], en[1], en[2]};
            if (z >= nz) e1[0] = e1[1] = e1[2] = zero4();  // E beyond the high face reads as zero
            float t[6][4];  // curl terms: Hx (1,2), Hy (3,4), Hz (5,6)
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const float ezp = m < 3 ? ec[2].v[m + 1] : ez_ip, eyp = m < 3 ? ec[1].v[m + 1] : ey_ip;
                t[0][m] = (ez_jp.v[m] - ec[2].v[m]) * ry;   // dEz/dy
                t[1][m] = (e1[1].v[m] - ec[1].v[m]) * rz;   // dEy/dz
                t[2][m] = (e1[0].v[m] - ec[0].v[m]) * rz;   // dEx/dz
                t[3][m] = (ezp - ec[2].v[m]) * rx;          // dEz/dx
                t[4][m] = (eyp - ec[1].v[m]) * rx;          // dEy/dx
                t[5][m] = (ex_jp.v[m] - ec[0].v[m]) * ry;   // dEx/dy
            }
            const bool all[4] = {true, true, true, true};
            if (XS && sx >= 0) {  // x slab: Hy's d/dx Ez, Hz's d/dx Ey
                const V4 bm = ld4(&S.prx[3][li]), aa = ld4(&S.prx[4][li]), ik = ld4(&S.prx[5][li]);
                float d3[4], d4[4];
#pragma unroll
                for (int m = 0; m < 4; m++) { d3[m] = t[3][m]; d4[m] = t[4][m]; }
                cterm4(t[3], ld4(S.phx[s] + pxo), a.psiHo[0][0], qHx, bm, aa, ik, d3, all, true);
                cterm4(t[4], ld4(S.phx[s] + pxc + pxo), a.psiHo[0][1], qHx, bm, aa, ik, d4, all, true);
            }
            if (YS && syb >= 0) {  // y slab: Hz's d/dy Ex, Hx's d/dy Ez
                const V4 bm = splat(S.pry[3][lj]), aa = splat(S.pry[4][lj]), ik = splat(S.pry[5][lj]);
                float d5[4], d0[4];
#pragma unroll
                for (int m = 0; m < 4; m++) { d5[m] = t[5][m]; d0[m] = t[0][m]; }
                cterm4(t[5], ld4(S.phy[s] + pyo), a.psiHo[1][0], qHy, bm, aa, ik, d5, all, true);
                cterm4(t[0], ld4(S.phy[s] + pyc + pyo), a.psiHo[1][1], qHy, bm, aa, ik, d0, all, true);
            }
            if (szh >= 0) {  // z slab: Hx's d/dz Ey, Hy's d/dz Ex
                const V4 bm = splat(S.pzp[3][q - 1]), aa = splat(S.pzp[4][q - 1]), ik = splat(S.pzp[5][q - 1]);
                float d1[4], d2[4];
#pragma unroll
                for (int m = 0; m < 4; m++) { d1[m] = t[1][m]; d2[m] = t[2][m]; }
                cterm4(t[1], pHz[0], a.psiHo[2][0], qHz, bm, aa, ik, d1, all, true);
                cterm4(t[2], pHz[1], a.psiHo[2][1], qHz, bm, aa, ik, d2, all, true);
            }
            V4 hn[3];
#pragma unroll
            for (int m = 0; m < 4; m++) {
                hn[0].v[m] = hb[0].v[m] - cH * (t[0][m] - t[1][m]);
                hn[1].v[m] = hb[1].v[m] - cH * (t[2][m] - t[3][m]);
                hn[2].v[m] = hb[2].v[m] - cH * (t[4][m] - t[5][m]);
            }
#pragma unroll
            for (int c = 0; c < 3; c++) {
                st4(a.Ho[c] + chh, hn[c]);
                st4(a.Eo[c] + chh, ec[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            hb[c] = hc[c];
            ec[c] = en[c];
        }
        hbh_x = hch_x;
    }
    if (S.abort_flag) {
        if (threadIdx.x == 0) {
            atomicOr(a.err, DEVERR_WAIT);
            // the copies issued for planes q .. q+STAGES-1 may still be in
            // flight: wait for them (bounded) before the shared memory goes
            const int issued = min(np, q + STAGES);
            for (int qq = q; qq < issued; qq++)
                if (!mbar_wait(&S.bar[qq % STAGES], (qq / STAGES) & 1)) break;
        }
        __syncthreads();
    }
}

template <int K>
__global__ void __launch_bounds__(NT, K == 3 ? 2 : 3)
    k_fused(const __grid_constant__ FusedMaps maps, const __grid_constant__ FusedArgs a) {
    pdl_wait();
    fused_item<K, false>(a, maps.m, a.tiles[blockIdx.x % a.ntiles], (int)blockIdx.x / a.ntiles);
}

// A joint pass: item blockIdx.x of kind K of any instance; the instance's
// arguments are copied into shared memory, its maps read from the table
// (the host wrote them before the launch).
template <int K>
__global__ void __launch_bounds__(NT, K == 3 ? 2 : 3) k_fused_joint(const __grid_constant__ FusedJoint jt) {
    pdl_wait();
    Smem<K, true> &S = smem_of<K, true>();
    const int4 e = jt.items[K][blockIdx.x];
    const FusedInst &in = jt.tab[e.x];
    const int xb = in.par0 ^ jt.phase;
    const int4 *src = reinterpret_cast<const int4 *>(&in.a[xb]);
    int4 *dst = reinterpret_cast<int4 *>(&S.args);
    static_assert(sizeof(FusedArgs) % 16 == 0, "arguments copied in 16-byte pieces");
    for (int w = threadIdx.x; w < (int)(sizeof(FusedArgs) / 16); w += NT) dst[w] = src[w];
    const CUtensorMap *tm = in.maps[xb].m;
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; q++)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&tm[q]) : "memory");
    __syncthreads();
    fused_item<K, true>(S.args, tm, e.y, e.z);
}

// J_f of the listed tiles back to zero (the current of two steps ago).
__global__ void __launch_bounds__(TILE_X *TILE_Y *TILE_Z) k_jf_clear(Grid<float> g, JfSet j) {
    pdl_wait();
    pdl_release();
    const int count = *j.count;
    const int i0 = threadIdx.x % TILE_X, j0 = (threadIdx.x / TILE_X) % TILE_Y, k0 = threadIdx.x / (TILE_X * TILE_Y);
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const long long t = j.list[q];
        const int tx = (int)(t % g.nt[0]), ty = (int)((t / g.nt[0]) % g.nt[1]);
        const int tz = (int)(t / ((long long)g.nt[0] * g.nt[1]));
        const int i = tx * TILE_X + i0, jj = ty * TILE_Y + j0, k = tz * TILE_Z + k0;
        if (i >= g.n[0] || jj >= g.n[1] || k >= g.n[2]) continue;
        const long long e = ((long long)k * g.n[1] + jj) * g.n[0] + i;
#pragma unroll
        for (int c = 0; c < 3; c++) j.Jf[c][e] = 0.f;
    }
}

// The free-current term of Eq. 8 on the listed tiles, after the fused pass:
// dE = -cE J_f on every non-held edge; then its effect on the H^{n+3/2} the
// pass computed without it.  In H_h -= cH [ (1/k_a1 d_a1 E_a2 + psi) -
// (1/k_a2 d_a2 E_a1 + psi) ] the edge value E_c(p) enters the forward
// differences along each axis a != c at the H cells p (with -1/d_a) and
// p - e_a (with +1/d_a); with psi' = psi + ((b-1) psi + a dd) a change dd of
// a difference changes H_h by -cH sgn (1/kappa + a) dd and psi by a dd
// (profiles at the H position along a).  Cells shared with other edges or
// tiles take atomic adds.
__global__ void __launch_bounds__(TILE_X *TILE_Y *TILE_Z) k_jf_fix(Grid<float> g, FixArgs f) {
    pdl_wait();
    pdl_release();
    const int count = *f.jf.count;
    const int i0 = threadIdx.x % TILE_X, j0 = (threadIdx.x / TILE_X) % TILE_Y, k0 = threadIdx.x / (TILE_X * TILE_Y);
    const int L2 = 2 * g.L;
    for (int qt = blockIdx.x; qt < count; qt += gridDim.x) {
        const long long t = f.jf.list[qt];
        const int tx = (int)(t % g.nt[0]), ty = (int)((t / g.nt[0]) % g.nt[1]);
        const int tz = (int)(t / ((long long)g.nt[0] * g.nt[1]));
        const int p[3] = {tx * TILE_X + i0, ty * TILE_Y + j0, tz * TILE_Z + k0};
        if (p[0] >= g.n[0] || p[1] >= g.n[1] || p[2] >= g.n[2]) continue;
        const long long st[3] = {1, g.n[0], (long long)g.n[0] * g.n[1]};
        const long long e = p[2] * st[2] + p[1] * st[1] + p[0];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float jf = f.jf.Jf[c][e];
            const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
            if (jf == 0.f || p[a1] == 0 || p[a2] == 0) continue;  // no current, or a held edge
            const float dE = -f.cls_pack[f.ecls[c][e]].z * jf;
            f.E[c][e] += dE;
#pragma unroll
            for (int side = 0; side < 2; side++) {
                const int ax = side ? a2 : a1;      // derivative axis
                const int hcmp = 3 - c - ax;        // H component that takes d/d_ax E_c
                const float sgn = ((hcmp + 1) % 3 == ax) ? 1.f : -1.f;
                const int sidx = (hcmp - ax + 5) % 3;  // psi[ax][sidx] belongs to H_hcmp
#pragma unroll
                for (int lo = 0; lo < 2; lo++) {    // H cells p (lo = 0) and p - e_ax (lo = 1)
                    if (lo && p[ax] == 0) continue;
                    const int m = p[ax] - lo;
                    const float dd = (lo ? g.r[ax] : -g.r[ax]) * dE;
                    const float aa = f.aH[ax][m], ik = f.ikH[ax][m];
                    const long long hm = e - lo * st[ax];
                    atomicAdd(&f.H[hcmp][hm], -g.cH * sgn * (ik + aa) * dd);
                    const int sl = slab_of(g, ax, m);
                    if (sl >= 0) {
                        int q3[3] = {p[0], p[1], p[2]};
                        q3[ax] = m;
                        long long pq;
                        if (ax == 0) pq = ((long long)q3[2] * g.n[1] + q3[1]) * L2 + sl;
                        else if (ax == 1) pq = ((long long)q3[2] * L2 + sl) * g.n[0] + q3[0];
                        else pq = ((long long)sl * g.n[1] + q3[1]) * g.n[0] + q3[0];
                        atomicAdd(&f.psiH[ax][sidx][pq], aa * dd);
                    }
                }
            }
        }
    }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tensor map over the three components of a field ([3][nz][ny][nx] floats,
// components `cstride` bytes apart) with a box of bw x bh cells of one plane.
bool field_map(CUtensorMap *m, float *base, size_t cstride, const int n[3], int bw, int bh) {
    EncodeTiledFn enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2], 3};
    const cuuint64_t strides[3] = {(cuuint64_t)n[0] * 4, (cuuint64_t)n[0] * n[1] * 4, (cuuint64_t)cstride};
    const cuuint32_t box[4] = {(cuuint32_t)bw, (cuuint32_t)bh, 1, 3};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map over the two components of a slab memory (components `cstride`
// bytes apart): dims d0 x d1 x d2 floats, a box of b0 x b1 of one plane.
bool psi_map(CUtensorMap *m, float *base, size_t cstride, int d0, int d1, int d2, int b0, int b1) {
    EncodeTiledFn enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2, 2};
    const cuuint64_t strides[3] = {(cuuint64_t)d0 * 4, (cuuint64_t)d0 * d1 * 4, (cuuint64_t)cstride};
    const cuuint32_t box[4] = {(cuuint32_t)b0, (cuuint32_t)b1, 1, 2};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool fused_grid_ok(const Grid<float> &g) {
    if (g.n[0] % 4 != 0 || g.per[0] || g.per[1] || g.per[2]) return false;
    if (g.cpml[0] && g.L % 4 != 0) return false;  // a four-cell group lies in an x slab as a whole or not at all
    // a tile (with its halo column and row) meets the x or y slab of one face at most
    if ((g.cpml[0] || g.cpml[1]) && g.L > FUSED_MAX_L) return false;
    if (g.cpml[0] && g.n[0] <= TX + g.L) return false;
    if (g.cpml[1] && g.n[1] <= TY + g.L) return false;
    if ((unsigned long long)g.n[0] * g.n[1] * g.n[2] >= (1ull << 32)) return false;  // 32-bit cell offsets
    if (g.n[0] / TX >= 65536 || (g.n[1] + TY - 1) / TY >= 65536) return false;
    return encoder() != nullptr;
}

int fused_chunk(int nz, int inner_tiles, int sms) {
    // about eight waves of four blocks per SM over the inner tiles, in runs
    // of 8..MAX_CHUNK planes (each item also loads two planes beyond its run)
    const long long slots = 4LL * (sms > 0 ? sms : 152);
    const long long want = (8 * slots + inner_tiles - 1) / (inner_tiles > 0 ? inner_tiles : 1);
    long long chunk = (nz + want - 1) / (want > 0 ? want : 1);
    chunk = (chunk + 7) / 8 * 8;
    if (chunk < 8) chunk = 8;
    if (chunk > MAX_CHUNK) chunk = MAX_CHUNK;
    return (int)chunk;
}

int fused_slab_chunk(int chunk) {
    // On a grid with short inner runs (a small grid: few items in all), the
    // slab items, which take longer per plane, get half of that run (4
    // planes at least) so that more of them run at once: 128x64x64 27 against
    // 29 us per pass, 320x128x96 76 against 81.  Long runs stay (c3: 495
    // against 500 us with half).
    if (chunk >= 16) return chunk;
    const int c = chunk / 2 / 4 * 4;
    return c < 4 ? 4 : c;
}

int fused_tiles(const Grid<float> &g, std::vector<int> kinds[4]) {
    const int tx_n = (g.n[0] + TX - 1) / TX, ty_n = (g.n[1] + TY - 1) / TY;
    for (int k = 0; k < 4; k++) kinds[k].clear();
    auto touches = [&](int a, int lo, int hi) {  // cells lo..hi (inclusive) meet a slab of axis a
        if (!g.cpml[a]) return false;
        return lo < g.L || hi >= g.n[a] - g.L;
    };
    for (int ty = 0; ty < ty_n; ty++)
        for (int tx = 0; tx < tx_n; tx++) {
            // the tile and the halo row and column it computes E on
            const int k = (touches(0, tx * TX, tx * TX + TX) ? 2 : 0) | (touches(1, ty * TY, ty * TY + TY) ? 1 : 0);
            kinds[k].push_back(tx | (ty << 16));
        }
    return tx_n * ty_n;
}

bool fused_maps(FusedPlan &pl, const FusedBuf P[2], const int n[3], int L, const int cpml[3]) {
    for (int b = 0; b < 2; b++) {
        CUtensorMap *m = pl.maps[b].m;
        const size_t se = (size_t)((char *)P[b].E[1] - (char *)P[b].E[0]);
        const size_t sh = (size_t)((char *)P[b].H[1] - (char *)P[b].H[0]);
        if ((char *)P[b].E[2] - (char *)P[b].E[1] != (long)se || (char *)P[b].H[2] - (char *)P[b].H[1] != (long)sh)
            return false;
        if (se % 16 || sh % 16 || ((uintptr_t)P[b].E[0] & 15) || ((uintptr_t)P[b].H[0] & 15)) return false;
        if (!field_map(&m[0], P[b].E[0], se, n, EW, EH)) return false;
        if (!field_map(&m[1], P[b].H[0], sh, n, HW, HH)) return false;
        // x and y slab memory (the maps of an axis without slabs stay unused)
        for (int q = 2; q < 6; q++) m[q] = m[1];
        if (cpml[0]) {
            const size_t cs = (size_t)((char *)P[b].psiE[0][1] - (char *)P[b].psiE[0][0]);
            const size_t ch = (size_t)((char *)P[b].psiH[0][1] - (char *)P[b].psiH[0][0]);
            if (cs % 16 || ch % 16 || L > PXW || L % 4) return false;
            if (!psi_map(&m[2], P[b].psiE[0][0], cs, 2 * L, n[1], n[2], L, EH)) return false;
            if (!psi_map(&m[3], P[b].psiH[0][0], ch, 2 * L, n[1], n[2], L, EH)) return false;
        }
        if (cpml[1]) {
            const size_t cs = (size_t)((char *)P[b].psiE[1][1] - (char *)P[b].psiE[1][0]);
            const size_t ch = (size_t)((char *)P[b].psiH[1][1] - (char *)P[b].psiH[1][0]);
            const int rows = 2 * L < PYH ? 2 * L : PYH;
            if (cs % 16 || ch % 16 || L > PYH) return false;
            if (!psi_map(&m[4], P[b].psiE[1][0], cs, n[0], 2 * L, n[2], EW, rows)) return false;
            if (!psi_map(&m[5], P[b].psiH[1][0], ch, n[0], 2 * L, n[2], EW, rows)) return false;
        }
    }
    static std::once_flag once;
    static bool attr_ok = true;
    std::call_once(once, [] {
        auto set = [](const void *k, size_t bytes) {
            return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
        };
        attr_ok = set((const void *)k_fused<0>, smem_bytes<0, false>()) &&
                  set((const void *)k_fused<1>, smem_bytes<1, false>()) &&
                  set((const void *)k_fused<2>, smem_bytes<2, false>()) &&
                  set((const void *)k_fused<3>, smem_bytes<3, false>()) &&
                  set((const void *)k_fused_joint<0>, smem_bytes<0, true>()) &&
                  set((const void *)k_fused_joint<1>, smem_bytes<1, true>()) &&
                  set((const void *)k_fused_joint<2>, smem_bytes<2, true>()) &&
                  set((const void *)k_fused_joint<3>, smem_bytes<3, true>());
    });
    return attr_ok;
}

template <int K>
static void launch_kind(const FusedArgs &a, const FusedPlan &pl, int xbuf, int items, cudaStream_t s) {
    launch_pdl(k_fused<K>, dim3((unsigned)items), dim3(NT), smem_bytes<K, false>(), s, pl.maps[xbuf], a);
    launch_count() += 1;
}

void launch_fused_pass(const FusedArgs &base, const FusedPlan &pl, int xbuf, cudaStream_t s,
                       const cudaStream_t sk[3]) {
    int first[5] = {0};
    for (int k = 0; k < 4; k++) first[k + 1] = first[k] + pl.n_kind[k];
    FusedArgs a = base;
    // the slab kinds first, each on its own stream (their items take longer,
    // so their blocks are dispatched before the inner ones), the corner tiles
    // (two blocks per SM) before the x-slab and y-slab tiles; then the inner
    // tiles on s
    for (int k = 3; k >= 1; k--) {
        if (pl.n_kind[k] == 0) continue;
        a.tiles = pl.tiles + first[k];
        a.ntiles = pl.n_kind[k];
        a.chunk = pl.slab_chunk;
        const int items = pl.n_kind[k] * pl.slab_nchunks;
        if (k == 1) launch_kind<1>(a, pl, xbuf, items, sk[0]);
        else if (k == 2) launch_kind<2>(a, pl, xbuf, items, sk[1]);
        else launch_kind<3>(a, pl, xbuf, items, sk[2]);
    }
    if (pl.n_kind[0] > 0) {
        a.tiles = pl.tiles;
        a.ntiles = pl.n_kind[0];
        a.chunk = pl.chunk;
        launch_kind<0>(a, pl, xbuf, pl.n_kind[0] * pl.nchunks, s);
    }
}

template <int K>
static void launch_joint_kind(const FusedJoint &jt, cudaStream_t s) {
    if (jt.nitems[K] == 0) return;
    launch_pdl(k_fused_joint<K>, dim3((unsigned)jt.nitems[K]), dim3(NT), smem_bytes<K, true>(), s, jt);
    launch_count() += 1;
}

void launch_fused_joint(const FusedJoint &jt, cudaStream_t s, const cudaStream_t sk[3]) {
    launch_joint_kind<3>(jt, sk[2]);  // the slab kinds first, as for a single instance
    launch_joint_kind<2>(jt, sk[1]);
    launch_joint_kind<1>(jt, sk[0]);
    launch_joint_kind<0>(jt, s);
}

void launch_jf_clear(const Grid<float> &g, const JfSet &j, int max_tiles, cudaStream_t s) {
    int nblk = max_tiles < 4 * 152 ? max_tiles : 4 * 152;
    if (nblk < 1) nblk = 1;
    launch_pdl(k_jf_clear, dim3(nblk), dim3(TILE_X * TILE_Y * TILE_Z), 0, s, g, j);
    launch_count() += 1;
}

void launch_jf_fix(const Grid<float> &g, const FixArgs &f, int max_tiles, cudaStream_t s) {
    int nblk = max_tiles < 4 * 152 ? max_tiles : 4 * 152;
    if (nblk < 1) nblk = 1;
    launch_pdl(k_jf_fix, dim3(nblk), dim3(TILE_X * TILE_Y * TILE_Z), 0, s, g, f);
    launch_count() += 1;
}

}  // namespace pic
