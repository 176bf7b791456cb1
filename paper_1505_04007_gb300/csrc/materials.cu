// materials.cu -- per-edge material classes built on the device from the cell
// material map (what pic_create needs from the map, without a host pass over
// the grid).
//
// An E edge is shared by four cells (offsets -1 and 0 along the two axes
// transverse to it); its Drude coefficients (Eq. 6) and Ampere factor
// (Eq. 8) depend only on the multiset of their material ids, so the key of
// an edge is the four ids sorted ascending, packed one byte each.  Beyond a
// non-periodic face the cell index is clamped to the face, on a periodic
// axis it wraps.
//   k_edge_keys:    every distinct key of the grid (at most MAX_CLASSES), and
//                   whether a material id is out of range;
//   k_edge_classes: each edge's class = the position of its key among the
//                   sorted distinct keys, and per plane the smallest and
//                   largest class of its edges (equal: one class on the
//                   whole plane).
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr unsigned long long EMPTY = ~0ull;
constexpr int BLOCK_SET = 256;  // distinct keys one block collects before adding them to the grid's set

__device__ __forceinline__ int wrap_clamp(int x, int n, int per) {
    if (x < 0) return per ? x + n : 0;
    if (x >= n) return per ? x - n : n - 1;
    return x;
}

// Sorted key of the four cells around edge `comp` of cell (i, j, k).
__device__ __forceinline__ unsigned edge_key(const uint8_t *mat, const int n[3], const int per[3], int comp, int i,
                                             int j, int k) {
    const int a1 = (comp + 1) % 3, a2 = (comp + 2) % 3;
    unsigned id[4];
    int q = 0;
#pragma unroll
    for (int s1 = -1; s1 <= 0; s1++)
#pragma unroll
        for (int s2 = -1; s2 <= 0; s2++) {
            int p3[3] = {i, j, k};
            p3[a1] = wrap_clamp(p3[a1] + s1, n[a1], per[a1]);
            p3[a2] = wrap_clamp(p3[a2] + s2, n[a2], per[a2]);
            id[q++] = mat[((long long)p3[2] * n[1] + p3[1]) * n[0] + p3[0]];
        }
    // sort four values (a fixed network of five compare-exchanges)
#define CX(a, b) { const unsigned lo = min(id[a], id[b]), hi = max(id[a], id[b]); id[a] = lo; id[b] = hi; }
    CX(0, 1) CX(2, 3) CX(0, 2) CX(1, 3) CX(1, 2)
#undef CX
    return id[0] | id[1] << 8 | id[2] << 16 | id[3] << 24;
}

// Insert key into an open-addressing set of `cap` slots (a power of two);
// false when the set is full.
__device__ __forceinline__ bool set_insert(unsigned long long *set, int cap, unsigned key) {
    unsigned h = (key * 2654435761u) & (unsigned)(cap - 1);
    for (int probe = 0; probe < cap; probe++) {
        const unsigned long long old = atomicCAS(&set[h], EMPTY, (unsigned long long)key);
        if (old == EMPTY || old == (unsigned long long)key) return true;
        h = (h + 1) & (unsigned)(cap - 1);
    }
    return false;
}

// flags bit 0: more distinct keys than the set holds; bit 1: a material id >= n_materials
__global__ void __launch_bounds__(256) k_edge_keys(const uint8_t *mat, int nx, int ny, int nz, int px, int py, int pz,
                                                   int n_materials, unsigned long long *gset, int gcap, int *flags) {
    __shared__ unsigned long long bset[BLOCK_SET];
    __shared__ int bflag;
    for (int q = threadIdx.x; q < BLOCK_SET; q += blockDim.x) bset[q] = EMPTY;
    if (threadIdx.x == 0) bflag = 0;
    __syncthreads();
    const int n[3] = {nx, ny, nz}, per[3] = {px, py, pz};
    const long long N = (long long)nx * ny * nz;
    unsigned last = 0xffffffffu;  // skip repeats of this thread's last key (it was inserted already)
    bool have = false;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        if (mat[e] >= n_materials) atomicOr(&bflag, 2);
        const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long long)nx * ny));
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const unsigned key = edge_key(mat, n, per, c, i, j, k);
            if (have && key == last) continue;
            if (!set_insert(bset, BLOCK_SET, key)) atomicOr(&bflag, 1);
            last = key;
            have = true;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < BLOCK_SET; q += blockDim.x)
        if (bset[q] != EMPTY && !set_insert(gset, gcap, (unsigned)bset[q])) atomicOr(flags, 1);
    if (threadIdx.x == 0 && bflag) atomicOr(flags, bflag);
}

// class of every edge (position of its key in the sorted list) and the
// smallest / largest class per plane
__global__ void __launch_bounds__(256) k_edge_classes(const uint8_t *mat, int nx, int ny, int nz, int px, int py,
                                                      int pz, const unsigned *keys, int nkeys, uint8_t *ecls0,
                                                      uint8_t *ecls1, uint8_t *ecls2, int *pmin, int *pmax) {
    const int n[3] = {nx, ny, nz}, per[3] = {px, py, pz};
    uint8_t *out[3] = {ecls0, ecls1, ecls2};
    const long long plane = (long long)nx * ny;
    // blocks take whole planes in turn: one reduction per plane
    for (int k = blockIdx.x; k < nz; k += gridDim.x) {
        int lo = 0x7fffffff, hi = -1;
        for (long long r = threadIdx.x; r < plane; r += blockDim.x) {
            const int i = (int)(r % nx), j = (int)(r / nx);
            const long long e = k * plane + r;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const unsigned key = edge_key(mat, n, per, c, i, j, k);
                int a = 0, b = nkeys - 1;  // the key is in the list (k_edge_keys collected every key)
                while (a < b) {
                    const int m = (a + b) >> 1;
                    if (keys[m] < key) a = m + 1;
                    else b = m;
                }
                out[c][e] = (uint8_t)a;
                lo = min(lo, a);
                hi = max(hi, a);
            }
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&pmin[k], lo);
            atomicMax(&pmax[k], hi);
        }
    }
}

// n bytes from src (any memory the device can read: on a device with
// coherent access to pageable host memory, the caller's host array) to dst.
__global__ void __launch_bounds__(256) k_copy_bytes(const unsigned char *src, unsigned char *dst, long long n) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if ((((uintptr_t)src | (uintptr_t)dst) & 15) == 0) {
        const long long n16 = n / 16;
        for (long long q = t; q < n16; q += stride)
            reinterpret_cast<uint4 *>(dst)[q] = reinterpret_cast<const uint4 *>(src)[q];
        for (long long q = n16 * 16 + t; q < n; q += stride) dst[q] = src[q];
    } else {
        for (long long q = t; q < n; q += stride) dst[q] = src[q];
    }
}

}  // namespace

void launch_copy_bytes(const void *src, void *dst, long long n, cudaStream_t s) {
    if (n <= 0) return;
    long long nblk = (n / 16 + 255) / 256;
    if (nblk > 8 * 152) nblk = 8 * 152;
    if (nblk < 1) nblk = 1;
    k_copy_bytes<<<(unsigned)nblk, 256, 0, s>>>(static_cast<const unsigned char *>(src),
                                                static_cast<unsigned char *>(dst), n);
}

void launch_edge_keys(const uint8_t *mat, const int n[3], const int per[3], int n_materials, unsigned long long *gset,
                      int gcap, int *flags, cudaStream_t s) {
    const long long N = (long long)n[0] * n[1] * n[2];
    long long nblk = (N + 255) / 256;
    if (nblk > 8 * 152) nblk = 8 * 152;
    if (nblk < 1) nblk = 1;
    k_edge_keys<<<(unsigned)nblk, 256, 0, s>>>(mat, n[0], n[1], n[2], per[0], per[1], per[2], n_materials, gset, gcap,
                                               flags);
}

void launch_edge_classes(const uint8_t *mat, const int n[3], const int per[3], const unsigned *keys, int nkeys,
                         uint8_t *const ecls[3], int *pmin, int *pmax, cudaStream_t s) {
    const int nblk = n[2] < 8 * 152 ? n[2] : 8 * 152;
    k_edge_classes<<<nblk, 256, 0, s>>>(mat, n[0], n[1], n[2], per[0], per[1], per[2], keys, nkeys, ecls[0], ecls[1],
                                        ecls[2], pmin, pmax);
}

}  // namespace pic
