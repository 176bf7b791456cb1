// particles.cu -- electron push, charge-conserving current deposit, and the
// periodic brick sort that keeps neighbouring electrons in neighbouring
// threads.
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
//
// Deposit: a block first finds the bounding box of its electrons' stencil
// windows.  When the box fits in shared memory the block sums all of its
// contributions there (shared-memory atomics) and then adds each non-zero
// edge to J_f once; otherwise every contribution goes to J_f directly.  The
// brick sort (every SORT_EVERY steps, 4x4x4-cell bricks, frozen electrons
// last) keeps a block's electrons in a few bricks, so the box is small.
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

constexpr int PUSH_BLOCK = 256;
constexpr int DEP_SMEM_BYTES = 40 * 1024;  // stays under the 48 KB default with the static part

__device__ __forceinline__ long long tile_of(const int idx[3], const int nt[3]) {
    return ((long long)(idx[2] / TILE_Z) * nt[1] + idx[1] / TILE_Y) * nt[0] + idx[0] / TILE_X;
}

template <typename T>
__global__ void __launch_bounds__(PUSH_BLOCK) k_push_deposit(Grid<T> g, Fields<T> f, Particles<T> p, PushParams<T> pp) {
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
#pragma unroll
            for (int a = 0; a < 3; a++) p.bold[a][q] = gather(f.H[a], g, c1w, o1, STAG_H[a]);
            dep = pp.deposit != 0;
        }
    }

    // ---- deposit: bounding box of the block's stencil windows (nodes c0-1 .. c0+2)
    if (threadIdx.x < 3) {
        bb_lo[threadIdx.x] = 0x7fffffff;
        bb_hi[threadIdx.x] = -0x7fffffff;
    }
    __syncthreads();
    if (dep) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            atomicMin(&bb_lo[a], c0[a] - 1);
            atomicMax(&bb_hi[a], c0[a] + 2);
        }
    }
    __syncthreads();
    const int w0 = bb_hi[0] - bb_lo[0] + 1, w1 = bb_hi[1] - bb_lo[1] + 1, w2 = bb_hi[2] - bb_lo[2] + 1;
    const bool any = bb_hi[0] >= bb_lo[0];
    const long long vol = any ? (long long)w0 * w1 * w2 : 0;
    const bool in_smem = any && 3 * vol * (long long)sizeof(T) <= DEP_SMEM_BYTES;
    if (in_smem) {
        for (long long e = threadIdx.x; e < 3 * vol; e += blockDim.x) acc[e] = T(0);
        __syncthreads();
    }
    const int flagv = (int)(step + 1);
    if (dep) {
        // Esirkepov on the 4-node window base = c0-1.  The old shape covers
        // nodes 1..2 of the window, the new one nodes 1+sh..2+sh (sh = cell
        // shift, -1..1), so only nodes lo..hi carry weight; the cumulative
        // sum along the current's own axis is non-zero only on the edges
        // between them (exactly zero elsewhere, so those are not issued).
        T S0[3][4], dS[3][4];
        int base[3], lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int sh = c1[a] - c0[a];
            base[a] = c0[a] - 1;
            lo[a] = 1 + (sh < 0 ? sh : 0);
            hi[a] = 2 + (sh > 0 ? sh : 0);
            T S1[4];
            shape4(T(1) + o0[a], S0[a]);
            shape4(T(sh + 1) + o1[a], S1);
#pragma unroll
            for (int m = 0; m < 4; m++) dS[a][m] = S1[m] - S0[a][m];
        }
        const T third = T(1) / T(3);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
            T *J = f.Jf[c];
            for (int m2 = lo[a2]; m2 <= hi[a2]; m2++) {
                for (int m1 = lo[a1]; m1 <= hi[a1]; m1++) {
                    const T tr = S0[a1][m1] * S0[a2][m2] + T(0.5) * dS[a1][m1] * S0[a2][m2] +
                                 T(0.5) * S0[a1][m1] * dS[a2][m2] + third * dS[a1][m1] * dS[a2][m2];
                    if (tr == T(0)) continue;
                    int node[3];
                    node[a1] = base[a1] + m1;
                    node[a2] = base[a2] + m2;
                    T run = T(0);
                    for (int m0 = lo[c]; m0 < hi[c]; m0++) {
                        run += dS[c][m0] * tr;
                        node[c] = base[c] + m0;
                        const T v = pp.jscale[c] * run;
                        if (in_smem) {
                            const long long l = ((long long)(node[2] - bb_lo[2]) * w1 + (node[1] - bb_lo[1])) * w0 +
                                                (node[0] - bb_lo[0]);
                            atomicAdd(&acc[c * vol + l], v);
                        } else {
                            int idx[3];
#pragma unroll
                            for (int a = 0; a < 3; a++) idx[a] = wrap_or_clamp<T>(node[a], g.n[a], g.per[a]);
                            atomicAdd(&J[((long long)idx[2] * g.n[1] + idx[1]) * g.n[0] + idx[0]], v);
                            f.jf_flag[tile_of(idx, g.nt)] = flagv;
                        }
                    }
                }
            }
        }
    }
    if (in_smem) {
        __syncthreads();
        for (long long e = threadIdx.x; e < 3 * vol; e += blockDim.x) {
            const T v = acc[e];
            if (v == T(0)) continue;
            const int c = (int)(e / vol);
            const long long r = e - c * vol;
            int idx[3];
            idx[0] = wrap_or_clamp<T>(bb_lo[0] + (int)(r % w0), g.n[0], g.per[0]);
            idx[1] = wrap_or_clamp<T>(bb_lo[1] + (int)((r / w0) % w1), g.n[1], g.per[1]);
            idx[2] = wrap_or_clamp<T>(bb_lo[2] + (int)(r / ((long long)w0 * w1)), g.n[2], g.per[2]);
            atomicAdd(&f.Jf[c][((long long)idx[2] * g.n[1] + idx[1]) * g.n[0] + idx[0]], v);
            f.jf_flag[tile_of(idx, g.nt)] = flagv;
        }
    }
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

template <typename T>
void launch_push_deposit(const Grid<T> &g, const Fields<T> &f, const Particles<T> &p, const PushParams<T> &pp,
                         cudaStream_t s) {
    if (p.n <= 0) return;
    k_push_deposit<T><<<(unsigned)((p.n + PUSH_BLOCK - 1) / PUSH_BLOCK), PUSH_BLOCK, DEP_SMEM_BYTES, s>>>(g, f, p, pp);
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

template void launch_push_deposit<float>(const Grid<float> &, const Fields<float> &, const Particles<float> &,
                                         const PushParams<float> &, cudaStream_t);
template void launch_push_deposit<double>(const Grid<double> &, const Fields<double> &, const Particles<double> &,
                                          const PushParams<double> &, cudaStream_t);
template void launch_gather_bold<float>(const Grid<float> &, const Fields<float> &, const Particles<float> &,
                                        cudaStream_t);
template void launch_gather_bold<double>(const Grid<double> &, const Fields<double> &, const Particles<double> &,
                                         cudaStream_t);
template void launch_sort<float>(const Particles<float> &, const Particles<float> &, const SortBuffers &, cudaStream_t);
template void launch_sort<double>(const Particles<double> &, const Particles<double> &, const SortBuffers &,
                                  cudaStream_t);

}  // namespace pic
