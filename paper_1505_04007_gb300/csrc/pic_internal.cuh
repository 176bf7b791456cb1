// pic_internal.cuh -- device-side data views and kernel launchers shared by
// the translation units of libpic.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

namespace pic {

// An NVTX range over the rest of the enclosing scope, opened by every entry
// point of the C ABI (a no-op unless a timeline profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Tiles that carry the "free current was deposited here this step" flag.
constexpr int TILE_X = 32, TILE_Y = 4, TILE_Z = 4;
// Probe samples buffered on the device between DFT flushes (one graph).
constexpr int DFT_BLOCK = 64;
constexpr int MAX_SOURCES = 16;
// Electrons are re-sorted by 4x4x4-cell brick every SORT_EVERY steps (the
// default; a simulation may change it, to a divisor of DFT_BLOCK).
constexpr int SORT_BRICK = 4;
constexpr int SORT_EVERY = 16;
constexpr int SCAN_TILE = 4096;  // entries per block of the prefix scan

// Device error bits.
enum : int {
    DEVERR_JUMP = 1,             // a particle moved more than one cell in a step
    DEVERR_NONFINITE = 2,        // non-finite momentum in the pusher
    DEVERR_FIELD_NONFINITE = 4,  // a NaN or Inf in E or H (scan at pic_sync / pic_get_stats)
    DEVERR_WAIT = 8,             // a pipeline wait of the fused field pass ran out of time
};

// Grid geometry and scalar coefficients, passed by value to every kernel.
template <typename T>
struct Grid {
    int n[3];        // nx, ny, nz
    int per[3];      // axis is periodic
    int cpml[3];     // axis has absorbing slabs (psi storage exists)
    int L;           // slab thickness in cells
    T r[3];          // 1/dx, 1/dy, 1/dz
    T cH;            // dt/mu0
    int nt[3];       // flag tiles per axis
    long long ncell;
};

// The two field components that carry a derivative along axis a.
__host__ __device__ inline int psi_comp(int a, int s) { return (a + 1 + s) % 3; }

template <typename T>
struct Fields {
    T *E[3], *H[3], *Jp[3], *Jf[3];
    // psi[a][s]: derivative along axis a of the (a+1+s)%3 component's curl
    // term; compact storage over the 2L slab cells of axis a.
    T *psiH[3][2], *psiE[3][2];
    // CPML profiles: b-1, a and 1/kappa at integer (E) and half-integer (H)
    // positions; psi is advanced as psi += (b-1) psi + a dF.
    const T *bE[3], *aE[3], *ikE[3];
    const T *bH[3], *aH[3], *ikH[3];
    const uint8_t *ecls[3];           // edge class per E component
    const T *cls_kJm1, *cls_bJ, *cls_cE; // per-class Eq. 6 (kJ-1, bJ) and Eq. 8 factors
    const uint8_t *cls_metal;         // per-class: wp^2 > 0
    const float4 *cls_pack;           // per-class (kJ-1, bJ, cE, metal) in float (FP32 kernels)
    int *jf_flag;                     // per tile: step+1 when J_f was written
    int *jf_list;                     // tiles written this step (each once), for the J_f correction
    int *jf_count;                    // length of jf_list
    const long long *step;            // device step counter n
};

template <typename T>
struct Particles {
    int *cell[3];      // integer cell of the position
    T *off[3];         // offset within the cell, [0,1)
    T *u[3];           // gamma*v [m/s], leading part
    T *ulo[3];         // trailing part: gamma*v = u + ulo (compensated sum)
    T *bold[3];        // H^{n-1/2} gathered at x^n (carried from the last push)
    T *eg[3];          // E^n at x^n, gathered beside the H update
    uint8_t *status;   // 0 live, 1 frozen
    long long *id;     // input order
    long long n;
};

template <typename T>
struct PushParams {
    T qmdt2;        // q dt / (2 m)
    T inv_c2;       // 1/c^2
    T dtd[3];       // dt / d_a
    T mu0;
    T jscale[3];    // -q / (dt d_a1 d_a2) for the J_a deposit
    const uint8_t *mat;       // cell material id
    const uint8_t *mat_metal; // per material id: wp > 0
    int deposit;
    int dep_smem;   // largest node box (bytes, three components) a deposit block accumulates in shared memory
    int *err;
};
// Default of PushParams::dep_smem.  A block whose box is larger adds its
// contributions straight to J_f: clearing and flushing a large, mostly empty
// box (the sparse tails of a sorted bunch) costs more than the global atomics
// it saves (measured: 4 KB beats 2, 8, 16 and 40 KB, and direct-only, on the
// c2 step and on the 48-instance sweep).
constexpr int DEP_SMEM_DEFAULT = 4 * 1024;
constexpr int DEP_SMEM_MAX = 16 * 1024;

template <typename T>
struct Probes {
    int np, nf;
    unsigned mask;
    const double *xyz_cells;  // [np][3] positions in cell units
    const long long *st_idx;  // [np][3][8] grid index of each interpolation corner
    const T *st_w;            // [np][3][8] trilinear weight of each corner
    const double *freq;       // [nf]
    double *samples;          // [DFT_BLOCK][np][3]
    double *F;                // [np][3][nf][2]
    double *phasor;           // [DFT_BLOCK][nf][2]
    double dt;
};

// Counting-sort state: brick key per electron, per-brick counts (then
// offsets, then cursors) and the per-block partial sums of the scan.
struct SortBuffers {
    int nb[3];       // bricks per axis
    int nbricks;     // nb[0]*nb[1]*nb[2]; frozen electrons use key nbricks
    int *key;        // [max_particles]
    int *count;      // [nbricks + 1]
    int *part;       // [ceil((nbricks + 1) / SCAN_TILE)]
};

struct Source {
    int comp;
    int box[6];
    double amp, t0, tau, f0;
};

// Kernels launched on this host thread (every launcher adds its launches).
long long &launch_count();

// Record the message returned by pic_last_error() on this thread; returns code.
int set_last_error(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));

// ------------------------------------------------------------- field plan
// Boxes of cells for the FP32 four-cells-per-thread kernels (x bounds are
// multiples of 4).  cE is the Ampere factor of a box whose edges all share
// one non-metal material (used by the vacuum kernel only).
struct Box {
    int lo[3], hi[3];
    float cE;
};
constexpr int MAX_BOXES = 16;
struct BoxList {
    int n;
    Box b[MAX_BOXES];
    long long first[MAX_BOXES + 1];  // prefix sums of four-cell groups per box
};
// How the grid is cut for the FP32 field kernels: the interior box (no CPML
// slab) and the face boxes over the slabs (H), and the same partition cut by
// z-runs into planes of one uniform non-metal material (vac) and planes with
// metal or mixed materials (mat), inside and over the slabs (E).
struct FieldPlan {
    BoxList bulk, faces, vac, mat, fvac, fmat;
    int block = 256;  // threads per block of the interior vacuum kernels (bulk H, vac E): 128, 256 or 512
};
// FP32 four-cells-per-thread field kernels (nx % 4 == 0), fields_v4.cu
// bulk/interior boxes on s, boxes over the absorbing slabs on s2 (may be s)
void launch_v4_H(const Grid<float> &g, const Fields<float> &f, const FieldPlan &plan, cudaStream_t s, cudaStream_t s2);
// E: vacuum interior on s, absorbing-slab vacuum on s2, material interior on s3, absorbing-slab material on s4
void launch_v4_E(const Grid<float> &g, const Fields<float> &f, const FieldPlan &plan, cudaStream_t s, cudaStream_t s2,
                 cudaStream_t s3, cudaStream_t s4);
// plane_cls[k]: the class all edges of plane k share if it is non-metal, else
// 255.  Returns false when the grid does not suit these kernels.
bool make_field_plan(const Grid<float> &g, const uint8_t *plane_cls, const float *cls_cE, FieldPlan &p);

// ------------------------------------------------------- fused field pass
// (fields_fused.cu) FP32 grids with nx % 4 == 0 and no periodic axis: one
// pass computes E^{n+1} (without J_f) and H^{n+3/2}, reading the state at
// step n from one copy of the arrays and writing step n+1 to the other.
constexpr int FUSED_TX = 32, FUSED_TY = 15;  // tile of one work item (x, y)
constexpr int FUSED_MAX_L = 8;                 // thickest x or y absorbing slab the pass stages

// One copy of the state the pass reads or writes.
struct FusedBuf {
    float *E[3], *H[3], *Jp[3];
    float *psiE[3][2], *psiH[3][2];
};
// One step's free current and its tile bookkeeping (see mark_jf_tile).
struct JfSet {
    float *Jf[3];
    int *flag, *list, *count;
};
struct FusedArgs {
    Grid<float> g;
    float *Eo[3], *Ho[3];          // state at n+1 (written)
    const float *Jpi[3];           // Drude current at n-1/2 (read)
    float *Jpo[3];                 // ... at n+1/2 (written on metal edges)
    const float *psiEi[3][2];
    float *psiEo[3][2];
    const float *psiHi[3][2];
    float *psiHo[3][2];
    const float *bE[3], *aE[3], *ikE[3], *bH[3], *aH[3], *ikH[3];
    const uint8_t *ecls[3];
    const float4 *cls_pack;
    const float *plane_cE;         // per plane: cE of its one non-metal class, or -1 (per-edge classes)
    const int *tiles;              // packed tile indices (tx | ty << 16)
    int ntiles, chunk;             // tiles of this launch; planes per work item
    int *err;
};
// The six tensor maps of one input copy: E, H, and the x and y slab CPML
// memory (psi_E x, psi_H x, psi_E y, psi_H y).
struct FusedMaps {
    CUtensorMap m[6];
};
// One instance of a joint pass over several simulations (a device table
// entry): maps and arguments for reading copy 0 and copy 1; at phase p the
// pass reads copy par0 ^ p.
struct FusedInst {
    FusedMaps maps[2];
    FusedArgs a[2];
    int par0;
};
// A joint pass: the instance table and, per tile kind, the work items
// {instance, packed tile, chunk, 0} of every instance.
struct FusedJoint {
    const FusedInst *tab;
    const int4 *items[4];
    int nitems[4];
    int phase;
};
struct FixArgs {
    float *E[3], *H[3], *psiH[3][2];  // state at n+1 (corrected in place)
    JfSet jf;                         // this step's free current
    const uint8_t *ecls[3];
    const float4 *cls_pack;
    const float *aH[3], *ikH[3];
};
struct FusedPlan {
    FusedMaps maps[2];             // reading state copy 0 and 1
    // device: the tiles of the four kinds one after another (inner, y slab
    // only, x slab only, both), n_kind[k] of kind k
    const int *tiles = nullptr;
    int n_kind[4] = {0, 0, 0, 0};
    int chunk = 32, nchunks = 1;   // planes per item of the inner tiles, and items per tile column
    int slab_chunk = 8, slab_nchunks = 1;  // ... of the slab kinds (shorter runs: more of their items at once)
};
bool fused_grid_ok(const Grid<float> &g);
// Planes per work item for a grid of nz planes and inner_tiles tiles on a GPU with sms SMs.
int fused_chunk(int nz, int inner_tiles, int sms);
// Planes per work item of the slab kinds, given the inner tiles' run.
int fused_slab_chunk(int chunk);
// Tile lists of the pass by kind: bit 0 set when the tile (with its halo
// row) meets a y slab, bit 1 when it (with its halo column) meets an x slab.
// Returns the tile count.
int fused_tiles(const Grid<float> &g, std::vector<int> kinds[4]);
// Tensor maps of both state copies (E, H components equally spaced).
bool fused_maps(FusedPlan &pl, const FusedBuf P[2], const int n[3], int L, const int cpml[3]);
// The pass reading copy xbuf's maps: inner tiles on s, the y-slab, x-slab
// and corner kinds on sk[0], sk[1], sk[2] (launched first).
void launch_fused_pass(const FusedArgs &a, const FusedPlan &pl, int xbuf, cudaStream_t s, const cudaStream_t sk[3]);
// A joint pass (phase jt.phase) over the instances of jt: inner items on s,
// the y-slab, x-slab and corner kinds on sk[0], sk[1], sk[2] (launched first).
void launch_fused_joint(const FusedJoint &jt, cudaStream_t s, const cudaStream_t sk[3]);
void launch_jf_clear(const Grid<float> &g, const JfSet &j, int max_tiles, cudaStream_t s);
void launch_jf_fix(const Grid<float> &g, const FixArgs &f, int max_tiles, cudaStream_t s);

// Copy n bytes on the device from src (device memory, or host memory on a
// device that reads pageable host memory coherently) to dst (materials.cu).
void launch_copy_bytes(const void *src, void *dst, long long n, cudaStream_t s);
// Edge classes on the device (materials.cu).  launch_edge_keys adds every
// distinct sorted 4-cell key of the grid to gset (gcap slots of ~0: empty)
// and sets flags bit 0 when a set overflows, bit 1 when a material id is not
// below n_materials.  launch_edge_classes writes each edge's class (the
// position of its key in the ascending list keys) and per plane the smallest
// and largest class (pmin, pmax preset to INT_MAX-like / negative values).
void launch_edge_keys(const uint8_t *mat, const int n[3], const int per[3], int n_materials, unsigned long long *gset,
                      int gcap, int *flags, cudaStream_t s);
void launch_edge_classes(const uint8_t *mat, const int n[3], const int per[3], const unsigned *keys, int nkeys,
                         uint8_t *const ecls[3], int *pmin, int *pmax, cudaStream_t s);

// k-omega map of the probe line (probe.cu): out[q][f] = |sum_p F_p e^{-i k_q s_p}|^2.
void launch_probe_kw(const double *F, const double *xyz_cells, double cell, int axis, int np, int nf, int comp,
                     const double *k, int nk, double *out, cudaStream_t s);

// Mark tile t as holding free current of the step flagged v, and append it
// to the step's tile list the first time.
__device__ __forceinline__ void mark_jf_tile(int *flag, int *list, int *count, long long t, int v) {
    if (flag[t] != v && atomicExch(&flag[t], v) != v) list[atomicAdd(count, 1)] = (int)t;
}

// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while the kernel before it in the stream is still finishing.
// pdl_wait() blocks until that kernel has completed and its writes are
// visible (a no-op for a kernel launched normally), so it comes before any
// global memory access; pdl_release() then lets the next such kernel be
// scheduled early in turn (it still waits for this one to complete).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---------------------------------------------------------------- launchers
// Field updates; with a plan (FP32) the four-cells-per-thread kernels run,
// otherwise the one-cell-per-thread kernels of fields.cu.
template <typename T>
void launch_update_H(const Grid<T> &g, const Fields<T> &f, const FieldPlan *plan, cudaStream_t s, cudaStream_t s2);
template <typename T>
void launch_update_E(const Grid<T> &g, const Fields<T> &f, const FieldPlan *plan, cudaStream_t s, cudaStream_t s2,
                     cudaStream_t s3, cudaStream_t s4);
template <typename T>
void launch_gather_E(const Grid<T> &g, const Fields<T> &f, const Particles<T> &p, cudaStream_t s);
template <typename T>
void launch_jf_apply(const Grid<T> &g, const Fields<T> &f, int max_tiles, cudaStream_t s);
// Sets DEVERR_FIELD_NONFINITE in *err if any of the n values of E or H is a
// NaN or an Inf.
template <typename T>
void launch_nonfinite_scan(const Fields<T> &f, long long n, int *err, cudaStream_t s);
// Electrons [base, base + n) whose cell is metal, counted into *count (added to).
// The grid as the conversion of new electrons needs it.
struct ParticleIn {
    double d[3];
    int n[3], per[3];
};
// New electrons [base, base + n) from device copies of the caller's xyz and
// u (n x 3 doubles each, SI); counts[0] the rejected (non-finite or within
// two cells of a non-periodic face), counts[1] the others inside a metal.
template <typename T>
void launch_particles_in(const double *xyz, const double *u, long long n, long long base, const ParticleIn &in,
                         const Particles<T> &p, const uint8_t *mat, const uint8_t *mat_metal,
                         unsigned long long *counts, cudaStream_t s);

// gather_E: E^n is gathered at x^n in the same kernel (the fused field
// path) instead of read from the particles' eg array; H^{n-1/2}(x^n) comes
// from bold, and bold <- H^{n+1/2}(x^{n+1}) at the end, on both paths.
template <typename T>
void launch_push_deposit(const Grid<T> &g, const Fields<T> &f, const Particles<T> &p,
                         const PushParams<T> &pp, cudaStream_t s, bool gather_E = false);
template <typename T>
void launch_sort(const Particles<T> &p, const Particles<T> &scratch, const SortBuffers &sb, cudaStream_t s);
template <typename T>
void launch_gather_bold(const Grid<T> &g, const Fields<T> &f, const Particles<T> &p, cudaStream_t s);
template <typename T>
void launch_sources(const Grid<T> &g, const Fields<T> &f, const Source *src, int nsrc, double dt,
                    cudaStream_t s);
template <typename T>
void launch_step_tail(const Grid<T> &g, const Fields<T> &f, const Probes<T> &pr, long long *step,
                      cudaStream_t s);
template <typename T>
void launch_dft_flush(const Probes<T> &pr, const long long *step, int count, cudaStream_t s);

}  // namespace pic
