// api.cu -- host runtime behind the C ABI of include/pic.h.
//
// A handle owns one simulation instance on one device: a single arena of
// device memory (caller workspace or one cudaMalloc), the per-edge material
// classes (built on the device from the material map at create time) and
// CPML profiles, the particle and probe buffers, and a captured CUDA graph
// that replays DFT_BLOCK steps plus one probe-DFT flush.  Every entry point
// opens an NVTX range named after it, so that a timeline profiler shows the
// host side of each call beside the kernels it launched.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "../../include/pic.h"
#include "pic_internal.cuh"

using namespace pic;

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

namespace pic {
long long &launch_count() {
    static thread_local long long n = 0;
    return n;
}

int set_last_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}
}  // namespace pic

#define CUDA_TRY(expr)                                                                          \
    do {                                                                                        \
        cudaError_t _e = (expr);                                                                \
        if (_e != cudaSuccess) return fail(PIC_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
    } while (0)

// ------------------------------------------------------------------ arena --
struct Arena {
    char *base = nullptr;  // nullptr: sizing pass
    size_t used = 0;
    template <typename P>
    P *take(size_t count) {
        used = (used + 255) & ~size_t(255);
        P *p = base ? reinterpret_cast<P *>(base + used) : nullptr;
        used += count * sizeof(P);
        return p;
    }
};

static bool is_periodic(const pic_config *c, int a) { return c->bc[2 * a] == PIC_BC_PERIODIC; }
static bool has_cpml(const pic_config *c, int a) {
    return c->bc[2 * a] == PIC_BC_CPML || c->bc[2 * a + 1] == PIC_BC_CPML;
}

static int validate(const pic_config *c) {
    if (!c) return fail(PIC_ERR_ARG, "config is NULL");
    if (c->flags & ~(uint64_t)(PIC_FLAG_SPLIT_FIELDS | PIC_FLAG_STAGED_UPLOAD))
        return fail(PIC_ERR_ARG, "unknown flags 0x%llx", (unsigned long long)c->flags);
    if (c->precision != PIC_FP32 && c->precision != PIC_FP64) return fail(PIC_ERR_ARG, "unknown precision");
    const int64_t n[3] = {c->nx, c->ny, c->nz};
    const double d[3] = {c->dx, c->dy, c->dz};
    for (int a = 0; a < 3; a++) {
        if (n[a] < 1 || n[a] > (1 << 20)) return fail(PIC_ERR_ARG, "axis %d: %lld cells out of range", a, (long long)n[a]);
        if (!(d[a] > 0.0) || !std::isfinite(d[a])) return fail(PIC_ERR_ARG, "axis %d: bad cell size", a);
        int lo = c->bc[2 * a], hi = c->bc[2 * a + 1];
        if (lo < 0 || lo > 2 || hi < 0 || hi > 2) return fail(PIC_ERR_ARG, "axis %d: unknown boundary code", a);
        if ((lo == PIC_BC_PERIODIC) != (hi == PIC_BC_PERIODIC))
            return fail(PIC_ERR_ARG, "axis %d: periodic boundaries must be paired", a);
        if (has_cpml(c, a) && n[a] < 2 * (int64_t)c->cpml_cells + 4)
            return fail(PIC_ERR_ARG, "axis %d: %lld cells cannot hold two %d-cell CPML slabs", a, (long long)n[a],
                        c->cpml_cells);
    }
    if (c->ny > 4 * 65535LL || c->nz > 2 * 65535LL) return fail(PIC_ERR_UNSUPPORTED, "grid too tall for the launch shape");
    // cell offsets in 32 bits (the gathers); such a grid would not fit a GPU's memory anyway
    if ((unsigned long long)n[0] * n[1] * n[2] >= (1ull << 32)) return fail(PIC_ERR_UNSUPPORTED, "2^32 cells or more");
    if (c->cpml_cells < 1 && (has_cpml(c, 0) || has_cpml(c, 1) || has_cpml(c, 2)))
        return fail(PIC_ERR_ARG, "cpml_cells must be >= 1");
    if (!(c->dt > 0.0) || !(c->eps0 > 0.0) || !(c->mu0 > 0.0)) return fail(PIC_ERR_ARG, "dt, eps0, mu0 must be > 0");
    if (c->n_materials < 1 || c->n_materials > 256 || !c->materials || !c->material_id)
        return fail(PIC_ERR_ARG, "need 1..256 materials and a material map");
    double wpmax = 0.0;
    for (int m = 0; m < c->n_materials; m++) {
        const pic_material &mt = c->materials[m];
        if (!(mt.wp >= 0.0) || !(mt.gamma >= 0.0) || !(mt.eps_inf > 0.0))
            return fail(PIC_ERR_ARG, "material %d: need wp >= 0, gamma >= 0, eps_inf > 0", m);
        wpmax = std::max(wpmax, mt.wp);
    }
    const double c2 = 1.0 / (c->eps0 * c->mu0);
    const double s = 1.0 / (d[0] * d[0]) + 1.0 / (d[1] * d[1]) + 1.0 / (d[2] * d[2]);
    if (!(c2 * c->dt * c->dt * s + 0.25 * wpmax * wpmax * c->dt * c->dt < 1.0))
        return fail(PIC_ERR_CFL, "dt=%g violates c^2 dt^2 sum(1/d^2) + wp^2 dt^2/4 < 1", c->dt);
    if (c->max_particles < 0 || c->max_probes < 0 || c->max_freqs < 0) return fail(PIC_ERR_ARG, "negative capacity");
    if (c->max_probes > 20000) return fail(PIC_ERR_UNSUPPORTED, "max_probes above 20000");
    return PIC_OK;
}

// ---------------------------------------------------------------- the sim --
struct SimBase {
    virtual ~SimBase() {}
    // for pic_batch: the batch captures whole DFT_BLOCK-step blocks of its
    // instances into one graph
    virtual int batch_prepare() = 0;                  // pending host-side work (outside any capture)
    virtual bool batch_ready() const = 0;             // at a block boundary (no buffered samples)
    virtual long long launch_block_on(cudaStream_t from) = 0;  // one block on own streams, forked from `from`
    virtual void join_to(cudaStream_t to) = 0;                 // `to` waits for the block launched last
    virtual void after_block(long long kernels) = 0;  // host bookkeeping once the block is enqueued
    virtual long long graph_epoch() const = 0;        // changes whenever captured steps go stale
    virtual int step_direct(long long n) = 0;
    virtual cudaStream_t main_stream() const = 0;
    virtual int steps_to_boundary() const = 0;        // steps left in the current block (0 at a boundary)
    virtual long long cells() const = 0;
    virtual int set_tuning(const pic_tuning &t) = 0;
    virtual bool fused_capable() const = 0;  // the grid takes the fused field pass
    // joint fused pass of a batch (see Sim::joint_*)
    virtual bool joint_capable() const = 0;
    virtual void joint_entry(FusedInst &e, int chunk) const = 0;
    virtual void joint_items(int inst, int chunk, std::vector<int4> items[4]) const = 0;
    virtual int fused_chunk_planes() const = 0;
    virtual long long joint_pre(int s, cudaStream_t from) = 0;
    virtual long long joint_post(int s, cudaStream_t from) = 0;
    int device = -1;  // CUDA device the handle was created on
};

template <typename T>
struct Sim : SimBase {
    pic_config cfg{};
    int n[3];
    double d[3];
    long long N = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;  // electron kernels, beside the field updates
    cudaEvent_t ev_bfork = nullptr, ev_bjoin = nullptr;  // joins to a batch capture
    long long epoch = 0;          // bumped by drop_graph
    cudaStream_t aux = nullptr;   // field updates over the absorbing slabs, beside the interior ones
    cudaStream_t aux2 = nullptr, aux3 = nullptr;  // E over material planes (interior, slabs)
    cudaEvent_t ev_fork = nullptr, ev_gathered = nullptr, ev_h = nullptr, ev_join = nullptr;
    cudaEvent_t ev_hf = nullptr, ev_hj = nullptr, ev_ef = nullptr, ev_ej = nullptr, ev_ej2 = nullptr, ev_ej3 = nullptr;
    void *arena = nullptr;
    bool own_arena = false;
    size_t arena_bytes = 0;

    Grid<T> g{};
    Fields<T> f{};
    Particles<T> p{};
    Particles<T> psort{};  // scratch arrays the sort scatters into
    SortBuffers sb{};
    int sort_every = SORT_EVERY;  // a divisor of DFT_BLOCK
    int since_sort = SORT_EVERY;
    PushParams<T> pp{};
    Probes<T> pr{};
    uint8_t *d_mat = nullptr, *d_mat_metal = nullptr;
    // building the edge classes on the device: the distinct keys found, the
    // sorted key list, error flags, per-plane smallest / largest class
    static constexpr int KEYSET = 1024;
    unsigned long long *d_keyset = nullptr;
    unsigned *d_keys = nullptr;
    int *d_mflags = nullptr, *d_pmin = nullptr, *d_pmax = nullptr;
    uint8_t *d_ecls[3] = {nullptr, nullptr, nullptr};
    uint8_t *d_cls_metal = nullptr;
    float4 *d_cls_pack = nullptr;
    FieldPlan fplan{};
    bool use_plan = false;
    T *d_cls[3] = {nullptr, nullptr, nullptr};
    T *d_prof[18];
    int *d_flag = nullptr;
    int *d_jf_list = nullptr, *d_jf_count = nullptr;
    long long *d_step = nullptr;
    int *d_err = nullptr;
    double *d_probe_xyz = nullptr, *d_freq = nullptr, *d_samples = nullptr, *d_F = nullptr, *d_phasor = nullptr;
    long long *d_st_idx = nullptr;
    T *d_st_w = nullptr;
    size_t n_tiles = 0;
    int n_classes = 0;

    std::vector<Source> sources;
    long long step_host = 0;
    int buffered = 0;
    bool bold_stale = false;
    bool have_q = false;
    double q = 0, m = 0;
    // Fused FP32 field pass (fields_fused.cu): two copies of the field state
    // (P[0] are the arrays of f, P[1] the second copy) and two free-current
    // sets (J_f of even and odd steps; set 0 is f's).  While `fused_ready`,
    // at step count n the state of step n lives in copy n & 1 with H one
    // half step ahead (E^n, H^{n+1/2}, J_p^{n-1/2}, psi_E^n, psi_H^{n+1/2}),
    // copy (n + 1) & 1 holds H^{n-1/2} and psi_H^{n-1/2}, and J_f of the
    // last step is set (n - 1) & 1.  Otherwise the state is the plain one in
    // f (E^n, H^{n-1/2}, ...), as on the split path.
    bool fused_possible = false;  // the grid and flags take the fused pass (arena holds the second copy)
    // the device reads pageable host memory coherently (a Grace system): the
    // caller's host arrays are read by kernels directly instead of copied
    bool host_direct = false;
    bool fused = false;           // ... and its plan was built
    bool use_fused = true;        // launch setting: take the fused pass when `fused`
    bool fused_ready = false;
    FusedBuf P[2];
    JfSet jfs[2];
    FusedPlan fpl{};
    int *d_tiles = nullptr;
    std::vector<int> h_tiles;     // host copy of d_tiles
    float *d_plane_cE = nullptr;

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphExec_t gexec_odd = nullptr;  // fused: the block graph for blocks starting at an odd step
    long long graph_kernels = 0;   // kernels in one replay of the step graph
    // Captured runs shorter than a block: steps [pos, pos + len) of a block
    // entered with the sort counter at `since`, with the DFT flush when they
    // end the block.  A run of SEG_MIN steps or more is captured the second
    // time it is asked for (the first time it launches kernel by kernel:
    // capturing costs more than one run) and replayed from then on (the
    // SEG_CACHE most recently used are kept); shorter runs launch directly.
    struct Segment {
        int pos, len, since, par;
        cudaGraphExec_t exec;
        long long kernels, used;
    };
    std::vector<Segment> segs;
    long long seg_clock = 0;
    static constexpr int SEG_MIN = 8, SEG_CACHE = 16;
    long long kernels = 0;         // kernels launched by this simulation so far

    // all device buffers, in one pass; base == nullptr only measures
    void plan(Arena &a) {
        const size_t Ts = (size_t)N;
        // the three components of each field one after another, equally
        // spaced (the fused pass reads a field's three components with one
        // tensor copy)
        for (int c = 0; c < 3; c++) f.E[c] = a.take<T>(Ts);
        for (int c = 0; c < 3; c++) f.H[c] = a.take<T>(Ts);
        for (int c = 0; c < 3; c++) f.Jp[c] = a.take<T>(Ts);
        for (int c = 0; c < 3; c++) f.Jf[c] = a.take<T>(Ts);
        for (int ax = 0; ax < 3; ax++) {
            size_t slab = 0;
            if (g.cpml[ax]) slab = (size_t)(N / n[ax]) * 2 * cfg.cpml_cells;
            // the two components of each field's memory one after the other (one tensor copy reads both)
            for (int s = 0; s < 2; s++) f.psiH[ax][s] = slab ? a.take<T>(slab) : nullptr;
            for (int s = 0; s < 2; s++) f.psiE[ax][s] = slab ? a.take<T>(slab) : nullptr;
        }
        if constexpr (std::is_same<T, float>::value) {
            if (fused_possible) {  // the second copy of the state and the second free-current set
                FusedBuf &B = P[1];
                for (int c = 0; c < 3; c++) B.E[c] = a.take<float>(Ts);
                for (int c = 0; c < 3; c++) B.H[c] = a.take<float>(Ts);
                for (int c = 0; c < 3; c++) B.Jp[c] = a.take<float>(Ts);
                for (int c = 0; c < 3; c++) jfs[1].Jf[c] = a.take<float>(Ts);
                for (int ax = 0; ax < 3; ax++) {
                    const size_t slab = g.cpml[ax] ? (size_t)(N / n[ax]) * 2 * cfg.cpml_cells : 0;
                    for (int s = 0; s < 2; s++) B.psiH[ax][s] = slab ? a.take<float>(slab) : nullptr;
                    for (int s = 0; s < 2; s++) B.psiE[ax][s] = slab ? a.take<float>(slab) : nullptr;
                }
                jfs[1].flag = a.take<int>(n_tiles);
                jfs[1].list = a.take<int>(n_tiles);
                jfs[1].count = a.take<int>(1);
                const int ntl = ((n[0] + FUSED_TX - 1) / FUSED_TX) * ((n[1] + FUSED_TY - 1) / FUSED_TY);
                d_tiles = a.take<int>((size_t)ntl);
                d_plane_cE = a.take<float>((size_t)n[2]);
            }
        }
        for (int ax = 0; ax < 3; ax++)
            for (int q6 = 0; q6 < 6; q6++) d_prof[ax * 6 + q6] = a.take<T>(n[ax]);
        d_mat = a.take<uint8_t>(Ts);
        d_mat_metal = a.take<uint8_t>(256);
        d_keyset = a.take<unsigned long long>(KEYSET);
        d_keys = a.take<unsigned>(256);
        d_mflags = a.take<int>(1);
        d_pmin = a.take<int>((size_t)n[2]);
        d_pmax = a.take<int>((size_t)n[2]);
        for (int c = 0; c < 3; c++) d_ecls[c] = a.take<uint8_t>(Ts);
        for (int q3 = 0; q3 < 3; q3++) d_cls[q3] = a.take<T>(256);
        d_cls_metal = a.take<uint8_t>(256);
        d_cls_pack = a.take<float4>(256);
        d_flag = a.take<int>(n_tiles);
        d_jf_list = a.take<int>(n_tiles);
        d_jf_count = a.take<int>(1);
        d_step = a.take<long long>(1);
        d_err = a.take<int>(1);
        const size_t mp = (size_t)cfg.max_particles;
        for (int c = 0; c < 3; c++) {
            p.cell[c] = a.take<int>(mp);
            p.off[c] = a.take<T>(mp);
            p.u[c] = a.take<T>(mp);
            p.ulo[c] = a.take<T>(mp);
            p.bold[c] = a.take<T>(mp);
            p.eg[c] = a.take<T>(mp);
        }
        p.status = a.take<uint8_t>(mp);
        p.id = a.take<long long>(mp);
        for (int c = 0; c < 3; c++) {
            psort.cell[c] = a.take<int>(mp);
            psort.off[c] = a.take<T>(mp);
            psort.u[c] = a.take<T>(mp);
            psort.ulo[c] = a.take<T>(mp);
            psort.bold[c] = a.take<T>(mp);
        }
        psort.status = a.take<uint8_t>(mp);
        psort.id = a.take<long long>(mp);
        sb.key = a.take<int>(mp);
        sb.count = a.take<int>((size_t)sb.nbricks + 1);
        sb.part = a.take<int>(((size_t)sb.nbricks + 1 + SCAN_TILE - 1) / SCAN_TILE);
        const size_t npb = (size_t)cfg.max_probes, nfb = (size_t)cfg.max_freqs;
        d_probe_xyz = a.take<double>(3 * npb);
        d_st_idx = a.take<long long>(24 * npb);
        d_st_w = a.take<T>(24 * npb);
        d_freq = a.take<double>(nfb);
        d_samples = a.take<double>((size_t)DFT_BLOCK * npb * 3);
        d_F = a.take<double>(npb * 3 * nfb * 2);
        d_phasor = a.take<double>((size_t)DFT_BLOCK * nfb * 2);
    }

    void init_geometry(const pic_config *c) {
        cfg = *c;
        cfg.material_id = nullptr;
        cfg.materials = nullptr;
        n[0] = (int)c->nx; n[1] = (int)c->ny; n[2] = (int)c->nz;
        d[0] = c->dx; d[1] = c->dy; d[2] = c->dz;
        N = (long long)n[0] * n[1] * n[2];
        for (int a = 0; a < 3; a++) {
            g.n[a] = n[a];
            g.per[a] = is_periodic(c, a);
            g.cpml[a] = has_cpml(c, a);
            g.r[a] = (T)(1.0 / d[a]);
            g.nt[a] = (n[a] + (a == 0 ? TILE_X : a == 1 ? TILE_Y : TILE_Z) - 1) /
                      (a == 0 ? TILE_X : a == 1 ? TILE_Y : TILE_Z);
        }
        g.L = c->cpml_cells;
        g.cH = (T)(c->dt / c->mu0);
        g.ncell = N;
        n_tiles = (size_t)g.nt[0] * g.nt[1] * g.nt[2];
        for (int a = 0; a < 3; a++) sb.nb[a] = (n[a] + SORT_BRICK - 1) / SORT_BRICK;
        sb.nbricks = sb.nb[0] * sb.nb[1] * sb.nb[2];
        fused_possible = std::is_same<T, float>::value && !(c->flags & PIC_FLAG_SPLIT_FIELDS) && n[0] % 4 == 0 &&
                         !g.per[0] && !g.per[1] && !g.per[2] && (!g.cpml[0] || g.L % 4 == 0) &&
                         ((!g.cpml[0] && !g.cpml[1]) || g.L <= FUSED_MAX_L) &&
                         (!g.cpml[0] || n[0] > FUSED_TX + g.L) && (!g.cpml[1] || n[1] > FUSED_TY + g.L) &&
                         (long long)n[0] * n[1] * n[2] < (1LL << 32) && n[0] / FUSED_TX < 65536 &&
                         (n[1] + FUSED_TY - 1) / FUSED_TY < 65536;
    }

    // CPML grading at position pos (cell units) along axis a: b-1, a, 1/kappa.
    void profile(int a, double pos, double &b, double &aa, double &ik) const {
        const double L = cfg.cpml_cells;
        double rho = 0.0;
        if (g.cpml[a]) {
            if (cfg.bc[2 * a] == PIC_BC_CPML && pos < L) rho = L - pos;
            if (cfg.bc[2 * a + 1] == PIC_BC_CPML && pos > n[a] - L) rho = std::max(rho, pos - (n[a] - L));
        }
        if (rho <= 0.0) { b = 0.0; aa = 0.0; ik = 1.0; return; }
        const double eta0 = std::sqrt(cfg.mu0 / cfg.eps0);
        const double x = rho / L, xm = std::pow(x, cfg.cpml_order);
        const double sigma = cfg.cpml_sigma_fac * (cfg.cpml_order + 1.0) / (eta0 * d[a]) * xm;
        const double kappa = 1.0 + (cfg.cpml_kappa_max - 1.0) * xm;
        const double alpha = cfg.cpml_alpha_max * (1.0 - x);
        b = std::expm1(-(sigma / kappa + alpha) * cfg.dt / cfg.eps0);  // b - 1
        const double den = sigma * kappa + kappa * kappa * alpha;
        aa = (sigma > 0.0 && den > 0.0) ? sigma * b / den : 0.0;
        ik = 1.0 / kappa;
    }

    // Edge classes from the material map already on the device (materials.cu):
    // the distinct sorted 4-cell keys, numbered in ascending key order; their
    // Eq. 6 / Eq. 8 coefficients in FP64 on the host; every edge's class and
    // per plane whether all its edges share one non-metal class (plane_cls,
    // else 255).
    int device_classes(const pic_config *c, std::vector<T> cls[3], std::vector<uint8_t> &cls_metal,
                       std::vector<uint8_t> &plane_cls) {
        CUDA_TRY(cudaMemsetAsync(d_keyset, 0xff, KEYSET * sizeof(unsigned long long), stream));
        CUDA_TRY(cudaMemsetAsync(d_mflags, 0, sizeof(int), stream));
        CUDA_TRY(cudaMemsetAsync(d_pmin, 0x7f, (size_t)n[2] * sizeof(int), stream));
        CUDA_TRY(cudaMemsetAsync(d_pmax, 0x80, (size_t)n[2] * sizeof(int), stream));
        launch_edge_keys(d_mat, n, g.per, c->n_materials, d_keyset, KEYSET, d_mflags, stream);
        CUDA_TRY(cudaGetLastError());
        std::vector<unsigned long long> set(KEYSET);
        int flags = 0;
        CUDA_TRY(cudaMemcpyAsync(set.data(), d_keyset, KEYSET * sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(cudaMemcpyAsync(&flags, d_mflags, sizeof(int), cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(cudaStreamSynchronize(stream));
        if (flags & 2) return fail(PIC_ERR_ARG, "a material id is not below n_materials (%d)", c->n_materials);
        std::vector<unsigned> keys;
        for (unsigned long long v : set)
            if (v != ~0ull) keys.push_back((unsigned)v);
        if ((flags & 1) || keys.size() > 256) return fail(PIC_ERR_UNSUPPORTED, "more than 256 distinct edge materials");
        std::sort(keys.begin(), keys.end());
        for (int q3 = 0; q3 < 3; q3++) cls[q3].assign(256, (T)0);
        cls_metal.assign(256, 0);
        for (size_t cl = 0; cl < keys.size(); cl++) {
            double sw = 0, swg = 0, se = 0;
            for (int q4 = 0; q4 < 4; q4++) {
                const pic_material &mt = c->materials[(keys[cl] >> (8 * q4)) & 0xffu];
                sw += mt.wp * mt.wp;
                swg += mt.wp * mt.wp * mt.gamma;
                se += mt.eps_inf;
            }
            const double wp2 = sw / 4.0, gam = sw > 0 ? swg / sw : 0.0, einf = se / 4.0;
            const double dt = c->dt;
            cls[0][cl] = (T)(-2.0 * gam * dt / (2.0 + gam * dt));  // kJ - 1
            cls[1][cl] = (T)(2.0 * dt * c->eps0 * wp2 / (2.0 + gam * dt));
            cls[2][cl] = (T)(dt / (c->eps0 * einf));
            cls_metal[cl] = wp2 > 0.0;
        }
        n_classes = (int)keys.size();
        CUDA_TRY(cudaMemcpyAsync(d_keys, keys.data(), keys.size() * sizeof(unsigned), cudaMemcpyHostToDevice, stream));
        launch_edge_classes(d_mat, n, g.per, d_keys, (int)keys.size(), d_ecls, d_pmin, d_pmax, stream);
        CUDA_TRY(cudaGetLastError());
        std::vector<int> pmin(n[2]), pmax(n[2]);
        CUDA_TRY(cudaMemcpyAsync(pmin.data(), d_pmin, n[2] * sizeof(int), cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(cudaMemcpyAsync(pmax.data(), d_pmax, n[2] * sizeof(int), cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(cudaStreamSynchronize(stream));
        plane_cls.assign(n[2], 255);
        for (int k = 0; k < n[2]; k++)
            if (pmin[k] == pmax[k] && pmin[k] >= 0 && pmin[k] < 256 && !cls_metal[pmin[k]]) plane_cls[k] = (uint8_t)pmin[k];
        return PIC_OK;
    }

    int create(const pic_config *c) {
        CUDA_TRY(cudaGetDevice(&device));
        init_geometry(c);
        std::vector<uint8_t> cls_metal, plane_cls;
        std::vector<T> cls[3];
        int rc = PIC_OK;

        Arena sizing;
        plan(sizing);
        arena_bytes = sizing.used;
        if (c->workspace) {
            if (c->workspace_bytes < arena_bytes)
                return fail(PIC_ERR_OOM, "workspace of %zu bytes is below the %zu needed", c->workspace_bytes,
                            arena_bytes);
            if (((uintptr_t)c->workspace) & 255) return fail(PIC_ERR_ARG, "workspace must be 256-byte aligned");
            arena = c->workspace;
        } else {
            cudaError_t e = cudaMalloc(&arena, arena_bytes);
            if (e != cudaSuccess) {
                arena = nullptr;
                return fail(PIC_ERR_OOM, "cudaMalloc(%zu): %s", arena_bytes, cudaGetErrorString(e));
            }
            own_arena = true;
        }
        Arena real;
        real.base = (char *)arena;
        plan(real);

        if (c->stream) {
            stream = (cudaStream_t)c->stream;
        } else {
            CUDA_TRY(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
            own_stream = true;
        }
        CUDA_TRY(cudaMemsetAsync(arena, 0, arena_bytes, stream));
        {
            int least = 0, greatest = 0;
            CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
            CUDA_TRY(cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, greatest));
            CUDA_TRY(cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking));
            CUDA_TRY(cudaStreamCreateWithFlags(&aux2, cudaStreamNonBlocking));
            CUDA_TRY(cudaStreamCreateWithFlags(&aux3, cudaStreamNonBlocking));
            for (cudaEvent_t *e : {&ev_fork, &ev_gathered, &ev_h, &ev_join, &ev_hf, &ev_hj, &ev_ef, &ev_ej, &ev_ej2, &ev_ej3, &ev_bfork,
                                   &ev_bjoin})
                CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        }

        // material map and per-material metal flag (particle absorption), then the edge classes
        std::vector<uint8_t> metal(256, 0);
        for (int m2 = 0; m2 < c->n_materials; m2++) metal[m2] = c->materials[m2].wp > 0.0;
        {
            int pma = 0;
            CUDA_TRY(cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, device));
            host_direct = pma == 1 && !(c->flags & PIC_FLAG_STAGED_UPLOAD);
        }
        if (host_direct) {  // read where it is; done before any later return
            launch_copy_bytes(c->material_id, d_mat, N, stream);
            CUDA_TRY(cudaGetLastError());
            CUDA_TRY(cudaStreamSynchronize(stream));
        } else {
            CUDA_TRY(cudaMemcpyAsync(d_mat, c->material_id, (size_t)N, cudaMemcpyHostToDevice, stream));
        }
        CUDA_TRY(cudaMemcpyAsync(d_mat_metal, metal.data(), 256, cudaMemcpyHostToDevice, stream));
        rc = device_classes(c, cls, cls_metal, plane_cls);
        if (rc) return rc;
        for (int q3 = 0; q3 < 3; q3++)
            CUDA_TRY(cudaMemcpyAsync(d_cls[q3], cls[q3].data(), 256 * sizeof(T), cudaMemcpyHostToDevice, stream));
        std::vector<float4> pack(256);
        for (int q = 0; q < 256; q++)
            pack[q] = make_float4((float)cls[0][q], (float)cls[1][q], (float)cls[2][q], cls_metal[q] ? 1.f : 0.f);
        CUDA_TRY(cudaMemcpyAsync(d_cls_pack, pack.data(), 256 * sizeof(float4), cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemcpyAsync(d_cls_metal, cls_metal.data(), 256, cudaMemcpyHostToDevice, stream));
        // FP32 with whole four-cell groups per row: cut the grid for the
        // four-cells-per-thread kernels (planes of one non-metal material
        // take the kernel without per-edge material reads)
        if constexpr (std::is_same<T, float>::value) {
          if (n[0] % 4 == 0) {
            std::vector<float> cE(256);
            for (int q = 0; q < 256; q++) cE[q] = (float)cls[2][q];
            use_plan = make_field_plan(g, plane_cls.data(), cE.data(), fplan);
            fplan.block = 256;
            if (fused_possible) {
                for (int c = 0; c < 3; c++) {
                    P[0].E[c] = f.E[c];
                    P[0].H[c] = f.H[c];
                    P[0].Jp[c] = f.Jp[c];
                    jfs[0].Jf[c] = f.Jf[c];
                }
                for (int ax = 0; ax < 3; ax++)
                    for (int q2 = 0; q2 < 2; q2++) {
                        P[0].psiE[ax][q2] = f.psiE[ax][q2];
                        P[0].psiH[ax][q2] = f.psiH[ax][q2];
                    }
                jfs[0].flag = d_flag;
                jfs[0].list = d_jf_list;
                jfs[0].count = d_jf_count;
                std::vector<int> kinds[4];
                fused_tiles(g, kinds);
                std::vector<int> tiles;
                for (int k = 0; k < 4; k++) {
                    tiles.insert(tiles.end(), kinds[k].begin(), kinds[k].end());
                    fpl.n_kind[k] = (int)kinds[k].size();
                }
                std::vector<float> pce(n[2]);
                for (int k = 0; k < n[2]; k++) pce[k] = plane_cls[k] != 255 ? cE[plane_cls[k]] : -1.f;
                CUDA_TRY(cudaMemcpy(d_tiles, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice));
                h_tiles = tiles;
                CUDA_TRY(cudaMemcpy(d_plane_cE, pce.data(), pce.size() * sizeof(float), cudaMemcpyHostToDevice));
                fpl.tiles = d_tiles;
                int sms = 0;
                CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
                fpl.chunk = fused_chunk(n[2], fpl.n_kind[0], sms);
                fpl.nchunks = (n[2] + fpl.chunk - 1) / fpl.chunk;
                fpl.slab_chunk = fused_slab_chunk(fpl.chunk);
                fpl.slab_nchunks = (n[2] + fpl.slab_chunk - 1) / fpl.slab_chunk;
                fused = fused_grid_ok(g) && fused_maps(fpl, P, n, g.L, g.cpml);
            }
          }
        }
        // CPML profiles: per axis (b-1, a, 1/kappa) at E positions, then at H positions
        for (int a = 0; a < 3; a++) {
            std::vector<T> pf[6];
            for (auto &v : pf) v.resize(n[a]);
            for (int x = 0; x < n[a]; x++) {
                double b, aa, ik;
                profile(a, (double)x, b, aa, ik);
                pf[0][x] = (T)b; pf[1][x] = (T)aa; pf[2][x] = (T)ik;
                profile(a, x + 0.5, b, aa, ik);
                pf[3][x] = (T)b; pf[4][x] = (T)aa; pf[5][x] = (T)ik;
            }
            for (int q6 = 0; q6 < 6; q6++)
                CUDA_TRY(cudaMemcpyAsync(d_prof[a * 6 + q6], pf[q6].data(), n[a] * sizeof(T), cudaMemcpyHostToDevice,
                                         stream));
        }
        CUDA_TRY(cudaStreamSynchronize(stream));  // host staging vectors die at return

        for (int a = 0; a < 3; a++) {
            f.bE[a] = d_prof[a * 6 + 0]; f.aE[a] = d_prof[a * 6 + 1]; f.ikE[a] = d_prof[a * 6 + 2];
            f.bH[a] = d_prof[a * 6 + 3]; f.aH[a] = d_prof[a * 6 + 4]; f.ikH[a] = d_prof[a * 6 + 5];
            f.ecls[a] = d_ecls[a];
        }
        f.cls_kJm1 = d_cls[0]; f.cls_bJ = d_cls[1]; f.cls_cE = d_cls[2];
        f.cls_metal = d_cls_metal;
        f.cls_pack = d_cls_pack;
        f.jf_flag = d_flag;
        f.jf_list = d_jf_list;
        f.jf_count = d_jf_count;
        f.step = d_step;
        p.n = 0;
        pp.mat = d_mat;
        pp.mat_metal = d_mat_metal;
        pp.deposit = 1;
        pp.dep_smem = DEP_SMEM_DEFAULT;
        pp.err = d_err;
        pp.mu0 = (T)c->mu0;
        pp.inv_c2 = (T)(c->eps0 * c->mu0);
        for (int a = 0; a < 3; a++) pp.dtd[a] = (T)(c->dt / d[a]);
        pr.np = 0; pr.nf = 0; pr.mask = 0;
        pr.xyz_cells = d_probe_xyz; pr.st_idx = d_st_idx; pr.st_w = d_st_w; pr.freq = d_freq; pr.samples = d_samples; pr.F = d_F; pr.phasor = d_phasor;
        pr.dt = c->dt;
        return PIC_OK;
    }

    ~Sim() override {
        if (stream) cudaStreamSynchronize(stream);
        drop_graph();
        if (side) cudaStreamSynchronize(side);
        for (cudaStream_t x : {aux, aux2, aux3})
            if (x) cudaStreamSynchronize(x);
        if (own_arena && arena) cudaFree(arena);
        if (own_stream && stream) cudaStreamDestroy(stream);
        if (side) cudaStreamDestroy(side);
        for (cudaStream_t x : {aux, aux2, aux3})
            if (x) cudaStreamDestroy(x);
        for (cudaEvent_t e : {ev_fork, ev_gathered, ev_h, ev_join, ev_hf, ev_hj, ev_ef, ev_ej, ev_ej2, ev_ej3, ev_bfork, ev_bjoin})
            if (e) cudaEventDestroy(e);
    }

    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (gexec_odd) cudaGraphExecDestroy(gexec_odd);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        gexec_odd = nullptr;
        graph = nullptr;
        for (auto &sg : segs)
            if (sg.exec) cudaGraphExecDestroy(sg.exec);
        segs.clear();
        epoch++;
    }

    // ---------------------------------------------------- fused helpers --
    // f with E, H, J_p and the CPML memory of state copy b and free-current set j
    Fields<T> view(int b, int j) const {
        Fields<T> v = f;
        if constexpr (std::is_same<T, float>::value) {
            for (int c = 0; c < 3; c++) {
                v.E[c] = P[b].E[c];
                v.H[c] = P[b].H[c];
                v.Jp[c] = P[b].Jp[c];
                v.Jf[c] = jfs[j].Jf[c];
            }
            for (int ax = 0; ax < 3; ax++)
                for (int q2 = 0; q2 < 2; q2++) {
                    v.psiE[ax][q2] = P[b].psiE[ax][q2];
                    v.psiH[ax][q2] = P[b].psiH[ax][q2];
                }
            v.jf_flag = jfs[j].flag;
            v.jf_list = jfs[j].list;
            v.jf_count = jfs[j].count;
        }
        return v;
    }
    // The plain state at the current step count: E^n, H^{n-1/2}, J_p^{n-1/2}
    // and the last step's J_f (fused: from the copies that hold them).
    Fields<T> current() const {
        if (!fused_ready) return f;
        const int par = (int)(step_host & 1);
        Fields<T> v = view(par, par ^ 1);
        const Fields<T> o = view(par ^ 1, 0);
        for (int c = 0; c < 3; c++) v.H[c] = o.H[c];
        for (int ax = 0; ax < 3; ax++)
            for (int q2 = 0; q2 < 2; q2++) v.psiH[ax][q2] = o.psiH[ax][q2];
        return v;
    }

    // Enter the fused path's state at step count n from the plain one: copy
    // H^{n-1/2} (and psi_H) to copy 1, the rest of step n's state too when
    // n is odd, then H^{n+1/2} in copy n & 1 (the split H update); both
    // free-current sets start empty.
    int enter_fused() {
        if constexpr (std::is_same<T, float>::value) {
            if (!fused || !use_fused || fused_ready) return PIC_OK;
            const int par = (int)(step_host & 1);
            const size_t nb = (size_t)N * sizeof(float);
            for (int j = 0; j < 2; j++) {
                for (int c = 0; c < 3; c++) CUDA_TRY(cudaMemsetAsync(jfs[j].Jf[c], 0, nb, stream));
                CUDA_TRY(cudaMemsetAsync(jfs[j].flag, 0, n_tiles * sizeof(int), stream));
                CUDA_TRY(cudaMemsetAsync(jfs[j].count, 0, sizeof(int), stream));
            }
            auto dd = [&](float *dst, const float *src, size_t bytes) {
                return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, stream);
            };
            for (int c = 0; c < 3; c++) CUDA_TRY(dd(P[1].H[c], P[0].H[c], nb));
            for (int ax = 0; ax < 3; ax++)
                for (int q2 = 0; q2 < 2; q2++)
                    if (P[0].psiH[ax][q2]) CUDA_TRY(dd(P[1].psiH[ax][q2], P[0].psiH[ax][q2], slab_bytes(ax)));
            if (par) {
                for (int c = 0; c < 3; c++) {
                    CUDA_TRY(dd(P[1].E[c], P[0].E[c], nb));
                    CUDA_TRY(dd(P[1].Jp[c], P[0].Jp[c], nb));
                }
                for (int ax = 0; ax < 3; ax++)
                    for (int q2 = 0; q2 < 2; q2++)
                        if (P[0].psiE[ax][q2]) CUDA_TRY(dd(P[1].psiE[ax][q2], P[0].psiE[ax][q2], slab_bytes(ax)));
            }
            launch_update_H<T>(g, view(par, 0), use_plan ? &fplan : nullptr, stream, stream);
            CUDA_TRY(cudaGetLastError());
            fused_ready = true;
            drop_graph();
        }
        return PIC_OK;
    }

    // Back to the plain state in f (before E or H is overwritten): the last
    // step's J_f record is dropped (both sets cleared).
    int leave_fused() {
        if constexpr (std::is_same<T, float>::value) {
            if (!fused_ready) return PIC_OK;
            const int par = (int)(step_host & 1);
            const size_t nb = (size_t)N * sizeof(float);
            auto dd = [&](float *dst, const float *src, size_t bytes) {
                return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, stream);
            };
            if (par) {  // E^n, J_p, psi_E in copy 1 (H^{n-1/2} is in copy 0 already)
                for (int c = 0; c < 3; c++) {
                    CUDA_TRY(dd(P[0].E[c], P[1].E[c], nb));
                    CUDA_TRY(dd(P[0].Jp[c], P[1].Jp[c], nb));
                }
                for (int ax = 0; ax < 3; ax++)
                    for (int q2 = 0; q2 < 2; q2++)
                        if (P[0].psiE[ax][q2]) CUDA_TRY(dd(P[0].psiE[ax][q2], P[1].psiE[ax][q2], slab_bytes(ax)));
            } else {    // H^{n-1/2}, psi_H^{n-1/2} in copy 1
                for (int c = 0; c < 3; c++) CUDA_TRY(dd(P[0].H[c], P[1].H[c], nb));
                for (int ax = 0; ax < 3; ax++)
                    for (int q2 = 0; q2 < 2; q2++)
                        if (P[0].psiH[ax][q2]) CUDA_TRY(dd(P[0].psiH[ax][q2], P[1].psiH[ax][q2], slab_bytes(ax)));
            }
            for (int j = 0; j < 2; j++) {
                for (int c = 0; c < 3; c++) CUDA_TRY(cudaMemsetAsync(jfs[j].Jf[c], 0, nb, stream));
                CUDA_TRY(cudaMemsetAsync(jfs[j].flag, 0, n_tiles * sizeof(int), stream));
                CUDA_TRY(cudaMemsetAsync(jfs[j].count, 0, sizeof(int), stream));
            }
            fused_ready = false;

            drop_graph();
        }
        return PIC_OK;
    }
    size_t slab_bytes(int ax) const { return (size_t)(N / n[ax]) * 2 * cfg.cpml_cells * sizeof(T); }

    // One step on the fused path, from the state of step n in copy `par`
    // (= n & 1) to copy par ^ 1, on the main stream: J_f of the step before
    // last back to zero, the electrons' E^n, push and deposit into J_f set
    // `par` and the prescribed sources; then the fused pass (inner tiles on
    // the main stream, the three kinds of tiles over the x and y slabs on
    // aux, aux2, aux3); then the free-current correction and the probe
    // sample (fused_post).  pe (optional) receives timing events: 0 step
    // start, 2 and 3 push start and done, 8 pass start, 1 pass done, 4 and 5
    // correction start and done, 6 tail done.
    void launch_step_fused(bool sort, int par, cudaEvent_t *pe) {
        if constexpr (std::is_same<T, float>::value) {
            if (pe) cudaEventRecord(pe[0], stream);
            fused_pre(sort, par);
            // The push and the sources read E^n and H^{n+1/2} from copy par,
            // which the pass only reads, so they could run beside it; they run
            // before it: beside it the two share the SMs, and the step took as
            // long (616 against 621 us on c3) with the pass stretched by the
            // push's share.
            if (pe) cudaEventRecord(pe[2], stream);
            fused_push(par, stream);
            if (pe) cudaEventRecord(pe[3], stream);
            if (pe) cudaEventRecord(pe[8], stream);
            cudaEventRecord(ev_ef, stream);
            for (cudaStream_t x : {aux, aux2, aux3}) cudaStreamWaitEvent(x, ev_ef, 0);
            const cudaStream_t sk[3] = {aux, aux2, aux3};
            launch_fused_pass(fused_args(par), fpl, par, stream, sk);
            fork_join(aux, stream, ev_ej);
            fork_join(aux2, stream, ev_ej2);
            fork_join(aux3, stream, ev_ej3);
            if (pe) cudaEventRecord(pe[1], stream);
            fused_post(par, pe);
        }
    }
    // the brick sort and J_f of the step before last back to zero
    void fused_pre(bool sort, int par) {
        if constexpr (std::is_same<T, float>::value) {
            if (sort) {
                psort.n = p.n;
                launch_sort<T>(p, psort, sb, stream);
            }
            launch_jf_clear(g, jfs[par ^ 1], (int)n_tiles, stream);
        }
    }
    // the electrons' push and deposit into J_f set `par` (E^n, H^{n+1/2} from
    // copy par, H^{n-1/2} at x^n kept per electron) and the prescribed sources
    void fused_push(int par, cudaStream_t s) {
        if constexpr (std::is_same<T, float>::value) {
            const Fields<T> fx = view(par, par);
            if (p.n > 0) launch_push_deposit<T>(g, fx, p, pp, s, true);
            launch_sources<T>(g, fx, sources.data(), (int)sources.size(), cfg.dt, s);
        }
    }
    // the arguments of a fused pass reading copy xb and writing copy xb ^ 1
    FusedArgs fused_args(int xb) const {
        FusedArgs a{};
        if constexpr (std::is_same<T, float>::value) {
            const int yb = xb ^ 1;
            a.g = g;
            for (int c = 0; c < 3; c++) {
                a.Eo[c] = P[yb].E[c];
                a.Ho[c] = P[yb].H[c];
                a.Jpi[c] = P[xb].Jp[c];
                a.Jpo[c] = P[yb].Jp[c];
            }
            for (int ax = 0; ax < 3; ax++) {
                for (int q2 = 0; q2 < 2; q2++) {
                    a.psiEi[ax][q2] = P[xb].psiE[ax][q2];
                    a.psiEo[ax][q2] = P[yb].psiE[ax][q2];
                    a.psiHi[ax][q2] = P[xb].psiH[ax][q2];
                    a.psiHo[ax][q2] = P[yb].psiH[ax][q2];
                }
                a.bE[ax] = f.bE[ax]; a.aE[ax] = f.aE[ax]; a.ikE[ax] = f.ikE[ax];
                a.bH[ax] = f.bH[ax]; a.aH[ax] = f.aH[ax]; a.ikH[ax] = f.ikH[ax];
                a.ecls[ax] = f.ecls[ax];
            }
            a.cls_pack = f.cls_pack;
            a.plane_cE = d_plane_cE;
            a.chunk = fpl.chunk;
            a.err = d_err;
        }
        return a;
    }
    void fused_post(int par, cudaEvent_t *pe) {
        if constexpr (std::is_same<T, float>::value) {
            const int yb = par ^ 1;
            if (pe) cudaEventRecord(pe[4], stream);
            FixArgs fa{};
            for (int c = 0; c < 3; c++) {
                fa.E[c] = P[yb].E[c];
                fa.H[c] = P[yb].H[c];
                fa.ecls[c] = f.ecls[c];
                fa.aH[c] = f.aH[c];
                fa.ikH[c] = f.ikH[c];
                for (int q2 = 0; q2 < 2; q2++) fa.psiH[c][q2] = P[yb].psiH[c][q2];
            }
            fa.jf = jfs[par];
            fa.cls_pack = f.cls_pack;
            launch_jf_fix(g, fa, (int)n_tiles, stream);
            if (pe) cudaEventRecord(pe[5], stream);
            launch_step_tail<T>(g, view(yb, par ^ 1), pr, d_step, stream);
            if (pe) cudaEventRecord(pe[6], stream);
        }
    }

    // ---------------------------------------------------- joint fused pass --
    // In a batch, the fused passes of every instance that takes one run as a
    // single joint pass per step; each instance contributes its steps' work
    // before and after the pass, its table entry and its work items.
    bool joint_capable() const override { return fused && use_fused && fused_ready; }
    // (the joint pass has enough items to cut columns into fewer, longer
    // runs of planes than the instance alone: `chunk` planes per item)
    void joint_entry(FusedInst &e, int chunk) const override {
        for (int xb = 0; xb < 2; xb++) {
            e.maps[xb] = fpl.maps[xb];
            e.a[xb] = fused_args(xb);
            e.a[xb].chunk = chunk;
        }
        e.par0 = (int)(step_host & 1);
    }
    void joint_items(int inst, int chunk, std::vector<int4> items[4]) const override {
        const int nch = (n[2] + chunk - 1) / chunk;
        for (int k = 0, first = 0; k < 4; first += fpl.n_kind[k], k++)
            for (int c = 0; c < nch; c++)  // tile-major within each chunk, as a single pass orders them
                for (int t = 0; t < fpl.n_kind[k]; t++) items[k].push_back(make_int4(inst, h_tiles[first + t], c, 0));
    }
    int fused_chunk_planes() const override { return fpl.chunk; }
    // step s of a joint block: the work beside the pass, forked from `from`
    // (the sort and the J_f clear on the main stream, the push and the
    // sources on the high-priority side stream; joint_post orders the
    // correction after them)
    long long joint_pre(int s, cudaStream_t from) override {
        const long long before = launch_count();
        cudaEventRecord(ev_bfork, from);
        cudaStreamWaitEvent(stream, ev_bfork, 0);
        const int par = (int)((step_host + s) & 1);
        fused_pre(s % sort_every == 0, par);
        fork_join(stream, side, ev_fork);
        fused_push(par, side);
        fork_join(side, stream, ev_join);
        return launch_count() - before;
    }
    // ... and after it (the DFT flush after the block's last step)
    long long joint_post(int s, cudaStream_t from) override {
        const long long before = launch_count();
        cudaEventRecord(ev_bfork, from);
        cudaStreamWaitEvent(stream, ev_bfork, 0);
        fused_post((int)((step_host + s) & 1), nullptr);
        if (s == DFT_BLOCK - 1) launch_dft_flush<T>(pr, d_step, DFT_BLOCK, stream);
        return launch_count() - before;
    }

    // ------------------------------------------------------------ batch --
    int batch_prepare() override {
        int rc = enter_fused();
        return rc ? rc : refresh_bold();
    }
    bool batch_ready() const override { return buffered == 0; }
    long long launch_block_on(cudaStream_t from) override {
        const long long before = launch_count();
        cudaEventRecord(ev_bfork, from);
        cudaStreamWaitEvent(stream, ev_bfork, 0);
        launch_block();
        const long long k = launch_count() - before;
        launch_count() = before;  // captured, not launched
        return k;
    }
    void join_to(cudaStream_t to) override {
        cudaEventRecord(ev_bjoin, stream);
        cudaStreamWaitEvent(to, ev_bjoin, 0);
    }
    void after_block(long long k) override {
        kernels += k;
        step_host += DFT_BLOCK;
        since_sort = DFT_BLOCK - (DFT_BLOCK - 1) / sort_every * sort_every;  // steps since its last sort
    }
    long long graph_epoch() const override { return 2 * epoch + ((fused_ready && (step_host & 1)) ? 1 : 0); }
    int step_direct(long long n) override { return step(n); }
    int steps_to_boundary() const override { return buffered ? DFT_BLOCK - buffered : 0; }
    long long cells() const override { return N; }
    bool fused_capable() const override { return fused; }
    cudaStream_t main_stream() const override { return stream; }

    // DFT_BLOCK steps (a sort every sort_every, the first one included) and the DFT flush
    void launch_block() {
        const int par0 = (int)(step_host & 1);
        for (int s = 0; s < DFT_BLOCK; s++) launch_step(s % sort_every == 0, true, nullptr, (par0 + s) & 1);
        launch_dft_flush<T>(pr, d_step, DFT_BLOCK, stream);
    }

    // ---------------------------------------------------------- stepping --
    // Work queued on `to` after this waits for the work queued on `from` so far.
    static void fork_join(cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
        cudaEventRecord(ev, from);
        cudaStreamWaitEvent(to, ev, 0);
    }

    // One step.  On the side stream the electrons' E^n is gathered while
    // the main stream updates H (which leaves E alone); once H^{n+1/2} is
    // final the push and deposit run there while the main stream updates E
    // without the free current; k_jf_apply adds the free current once both
    // are done.  With concurrent = false everything runs in that order on
    // the main stream.  pe (optional) receives 7 timing events: step start,
    // H done, push start, push done, E start, E done, tail done.
    void launch_step(bool sort, bool concurrent = true, cudaEvent_t *pe = nullptr, int par = 0) {
        if (fused_ready) {
            launch_step_fused(sort, par, pe);
            return;
        }
        if (sort) {
            psort.n = p.n;
            launch_sort<T>(p, psort, sb, stream);
        }
        if (pe) cudaEventRecord(pe[0], stream);
        const bool parts = p.n > 0, fork = concurrent && parts;
        if (fork) {
            cudaEventRecord(ev_fork, stream);
            cudaStreamWaitEvent(side, ev_fork, 0);
            launch_gather_E<T>(g, f, p, side);
            cudaEventRecord(ev_gathered, side);
        } else if (parts) {
            launch_gather_E<T>(g, f, p, stream);
        }
        // the absorbing-slab boxes of each field update run on aux beside the interior boxes
        const bool split = concurrent && use_plan;
        if (split) fork_join(stream, aux, ev_hf);
        launch_update_H<T>(g, f, use_plan ? &fplan : nullptr, stream, split ? aux : stream);
        if (split) fork_join(aux, stream, ev_hj);
        if (pe) cudaEventRecord(pe[1], stream);
        launch_sources<T>(g, f, sources.data(), (int)sources.size(), cfg.dt, stream);
        if (fork) {
            cudaEventRecord(ev_h, stream);
            cudaStreamWaitEvent(side, ev_h, 0);
            if (pe) cudaEventRecord(pe[2], side);
            launch_push_deposit<T>(g, f, p, pp, side);
            if (pe) cudaEventRecord(pe[3], side);
            cudaEventRecord(ev_join, side);
            cudaStreamWaitEvent(stream, ev_gathered, 0);
        } else {
            if (pe) cudaEventRecord(pe[2], stream);
            if (parts) launch_push_deposit<T>(g, f, p, pp, stream);
            if (pe) cudaEventRecord(pe[3], stream);
        }
        if (pe) cudaEventRecord(pe[4], stream);
        if (split) {  // the four E pieces write disjoint cells: each on its own stream
            cudaEventRecord(ev_ef, stream);
            for (cudaStream_t x : {aux, aux2, aux3}) cudaStreamWaitEvent(x, ev_ef, 0);
        }
        launch_update_E<T>(g, f, use_plan ? &fplan : nullptr, stream, split ? aux : stream, split ? aux2 : stream,
                           split ? aux3 : stream);
        if (split) {
            fork_join(aux, stream, ev_ej);
            fork_join(aux2, stream, ev_ej2);
            fork_join(aux3, stream, ev_ej3);
        }
        if (pe) cudaEventRecord(pe[5], stream);
        if (fork) cudaStreamWaitEvent(stream, ev_join, 0);
        launch_jf_apply<T>(g, f, (int)n_tiles, stream);
        launch_step_tail<T>(g, f, pr, d_step, stream);
        if (pe) cudaEventRecord(pe[6], stream);
    }

    // The block graph for a block starting at the current step count (on
    // the fused path blocks starting at odd steps have their own graph).
    int ensure_graph(cudaGraphExec_t **out = nullptr) {
        cudaGraphExec_t &slot = (fused_ready && (step_host & 1)) ? gexec_odd : gexec;
        if (out) *out = &slot;
        if (slot) return PIC_OK;
        CUDA_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        const long long before = launch_count();
        launch_block();
        graph_kernels = launch_count() - before;
        launch_count() = before;  // captured, not launched
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamEndCapture(stream, &gr);
        if (e != cudaSuccess) return fail(PIC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&slot, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) { slot = nullptr; return fail(PIC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
        return PIC_OK;
    }

    // Replay (capturing it the first time) the run of len steps from the
    // current position in the block; the host counters advance as the
    // direct path would advance them.
    int run_segment(int len) {
        const int pos = buffered, since = std::min(since_sort, sort_every);
        const int par0 = fused_ready ? (int)(step_host & 1) : 0;
        const bool ends = pos + len == DFT_BLOCK;
        Segment *sg = nullptr;
        for (auto &x : segs)
            if (x.pos == pos && x.len == len && x.since == since && x.par == par0) sg = &x;
        if (!sg) {  // first use: remember it and launch directly
            if ((int)segs.size() >= SEG_CACHE) {
                size_t old = 0;
                for (size_t q = 1; q < segs.size(); q++)
                    if (segs[q].used < segs[old].used) old = q;
                if (segs[old].exec) cudaGraphExecDestroy(segs[old].exec);
                segs.erase(segs.begin() + (long)old);
            }
            segs.push_back(Segment{pos, len, since, par0, nullptr, 0, ++seg_clock});
            return run_direct(len);
        }
        if (!sg->exec) {
            Segment nsg{pos, len, since, par0, nullptr, 0, 0};
            CUDA_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
            const long long before = launch_count();
            int ss = since;
            for (int q = 0; q < len; q++) {
                const bool sort = ss >= sort_every;
                launch_step(sort, true, nullptr, (par0 + q) & 1);
                ss = sort ? 1 : ss + 1;
            }
            if (ends) launch_dft_flush<T>(pr, d_step, DFT_BLOCK, stream);
            nsg.kernels = launch_count() - before;
            launch_count() = before;  // captured, not launched
            cudaGraph_t gr = nullptr;
            cudaError_t e = cudaStreamEndCapture(stream, &gr);
            if (e != cudaSuccess) return fail(PIC_ERR_CUDA, "segment capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&nsg.exec, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) return fail(PIC_ERR_CUDA, "segment instantiate: %s", cudaGetErrorString(e));
            sg->exec = nsg.exec;
            sg->kernels = nsg.kernels;
        }
        sg->used = ++seg_clock;
        CUDA_TRY(cudaGraphLaunch(sg->exec, stream));
        kernels += sg->kernels;
        int ss = since;
        for (int q = 0; q < len; q++) ss = ss >= sort_every ? 1 : ss + 1;
        since_sort = ss;
        step_host += len;
        buffered = ends ? 0 : pos + len;
        return PIC_OK;
    }

    int refresh_bold() {
        if (bold_stale) {
            launch_gather_bold<T>(g, current(), p, stream);
            CUDA_TRY(cudaGetLastError());
            bold_stale = false;
        }
        return PIC_OK;
    }

    int step(long long nsteps) {
        if (nsteps < 0) return fail(PIC_ERR_ARG, "negative step count");
        const long long direct0 = launch_count();
        int rc = step_inner(nsteps);
        kernels += launch_count() - direct0;
        return rc;
    }

    int prepare() {
        int rc = enter_fused();
        return rc ? rc : refresh_bold();
    }

    int step_inner(long long nsteps) {
        int rc = nsteps > 0 ? prepare() : refresh_bold();
        if (rc) return rc;
        while (nsteps > 0) {
            if (buffered == 0 && nsteps >= DFT_BLOCK) {
                cudaGraphExec_t *ex = nullptr;
                rc = ensure_graph(&ex);
                if (rc) return rc;
                CUDA_TRY(cudaGraphLaunch(*ex, stream));
                kernels += graph_kernels;
                nsteps -= DFT_BLOCK;
                step_host += DFT_BLOCK;
                since_sort = DFT_BLOCK - (DFT_BLOCK - 1) / sort_every * sort_every;  // steps since its last sort
                continue;
            }
            const int run = (int)std::min<long long>(nsteps, DFT_BLOCK - buffered);
            if (run >= SEG_MIN) {  // a captured run up to the end of the block, or the last steps asked for
                rc = run_segment(run);
                if (rc) return rc;
                nsteps -= run;
                continue;
            }
            rc = run_direct(1);
            if (rc) return rc;
            nsteps--;
        }
        CUDA_TRY(cudaGetLastError());
        return PIC_OK;
    }

    // len steps launched kernel by kernel (within the current block)
    int run_direct(int len) {
        for (int q = 0; q < len; q++) {
            const bool sort = since_sort >= sort_every;
            launch_step(sort, true, nullptr, (int)(step_host & 1));
            since_sort = sort ? 1 : since_sort + 1;
            CUDA_TRY(cudaGetLastError());
            buffered++;
            step_host++;
            if (buffered == DFT_BLOCK) {
                launch_dft_flush<T>(pr, d_step, DFT_BLOCK, stream);
                buffered = 0;
            }
        }
        return PIC_OK;
    }

    int flush_probes() {
        if (buffered > 0) {
            launch_dft_flush<T>(pr, d_step, buffered, stream);
            CUDA_TRY(cudaGetLastError());
            buffered = 0;
        }
        return PIC_OK;
    }

    int sync() {
        CUDA_TRY(cudaStreamSynchronize(stream));
        int err = 0;
        CUDA_TRY(cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (err & (DEVERR_JUMP | DEVERR_NONFINITE | DEVERR_WAIT))
            return fail(PIC_ERR_DEVICE, "kernel error bits 0x%x%s%s", err,
                        (err & DEVERR_NONFINITE) ? " (non-finite electron momentum: those electrons are frozen)" : "",
                        (err & DEVERR_WAIT) ? " (a wait of the fused field pass ran out of time)" : "");
        if (err & DEVERR_FIELD_NONFINITE) return fail(PIC_ERR_NONFINITE, "E or H holds a NaN or an Inf");
        return PIC_OK;
    }

    // sync() after a scan of E and H for NaN or Inf (pic_sync, pic_get_stats)
    int check() {
        CUDA_TRY(cudaStreamSynchronize(stream));
        launch_nonfinite_scan<T>(current(), N, d_err, stream);
        CUDA_TRY(cudaGetLastError());
        return sync();
    }

    // ------------------------------------------------------ checkpoint --
    // File: magic, fixed header (geometry, precision, arena size, host-side
    // counters), the source list, then the whole device arena.  The arena's
    // layout is a function of the configuration alone, so a handle created
    // with the same configuration restores every array exactly.
    struct SaveHeader {
        char magic[8];
        uint32_t version;
        int32_t precision;
        int64_t n[3];
        uint64_t arena_bytes;
        int64_t max_particles;
        int32_t max_probes, max_freqs;
        int64_t step_host, np;
        int32_t buffered, since_sort, bold_stale, have_q, deposit, probe_np, probe_nf, nsources;
        uint32_t probe_mask, pad;
        double q, m;
        // configuration scalars (compared on load; the configuration's arrays
        // are compared byte by byte with the file's copy of them)
        double d[3], dt, eps0, mu0;
        int32_t bc[6], cpml_cells, pad2;
        double cpml_order, cpml_sigma_fac, cpml_kappa_max, cpml_alpha_max;
        uint64_t flags;
        int32_t fused_ready, pad3;
    };

    // Arena pieces that follow from the configuration alone (material map,
    // edge classes and their coefficients, CPML profiles): (offset, bytes).
    std::vector<std::pair<size_t, size_t>> config_regions() const {
        std::vector<std::pair<size_t, size_t>> r;
        auto add = [&](const void *ptr, size_t bytes) { r.emplace_back((size_t)((const char *)ptr - (const char *)arena), bytes); };
        add(d_mat, (size_t)N);
        add(d_mat_metal, 256);
        for (int c = 0; c < 3; c++) add(d_ecls[c], (size_t)N);
        for (int q3 = 0; q3 < 3; q3++) add(d_cls[q3], 256 * sizeof(T));
        add(d_cls_metal, 256);
        add(d_cls_pack, 256 * sizeof(float4));
        for (int a = 0; a < 3; a++)
            for (int q6 = 0; q6 < 6; q6++) add(d_prof[a * 6 + q6], (size_t)n[a] * sizeof(T));
        return r;
    }

    int save(const char *path) {
        int rc = sync();
        if (rc) return rc;
        SaveHeader hd{};
        memcpy(hd.magic, "PICSAVE1", 8);
        hd.version = 2;
        for (int a = 0; a < 3; a++) hd.d[a] = d[a];
        hd.dt = cfg.dt;
        hd.eps0 = cfg.eps0;
        hd.mu0 = cfg.mu0;
        for (int q6 = 0; q6 < 6; q6++) hd.bc[q6] = cfg.bc[q6];
        hd.cpml_cells = cfg.cpml_cells;
        hd.cpml_order = cfg.cpml_order;
        hd.cpml_sigma_fac = cfg.cpml_sigma_fac;
        hd.cpml_kappa_max = cfg.cpml_kappa_max;
        hd.cpml_alpha_max = cfg.cpml_alpha_max;
        hd.flags = cfg.flags;
        hd.fused_ready = fused_ready ? 1 : 0;
        hd.precision = cfg.precision;
        for (int a = 0; a < 3; a++) hd.n[a] = n[a];
        hd.arena_bytes = arena_bytes;
        hd.max_particles = cfg.max_particles;
        hd.max_probes = cfg.max_probes;
        hd.max_freqs = cfg.max_freqs;
        hd.step_host = step_host;
        hd.np = p.n;
        hd.buffered = buffered;
        hd.since_sort = since_sort;
        hd.bold_stale = bold_stale;
        hd.have_q = have_q;
        hd.deposit = pp.deposit;
        hd.probe_np = pr.np;
        hd.probe_nf = pr.nf;
        hd.probe_mask = pr.mask;
        hd.nsources = (int)sources.size();
        hd.q = q;
        hd.m = m;
        FILE *fp = fopen(path, "wb");
        if (!fp) return fail(PIC_ERR_ARG, "cannot open %s for writing", path);
        bool ok = fwrite(&hd, sizeof hd, 1, fp) == 1;
        if (ok && !sources.empty()) ok = fwrite(sources.data(), sizeof(Source), sources.size(), fp) == sources.size();
        std::vector<char> buf;
        const size_t chunk = (size_t)64 << 20;
        for (size_t off = 0; ok && off < arena_bytes; off += chunk) {
            const size_t len = std::min(chunk, arena_bytes - off);
            buf.resize(len);
            if (cudaMemcpy(buf.data(), (char *)arena + off, len, cudaMemcpyDeviceToHost) != cudaSuccess) {
                fclose(fp);
                return fail(PIC_ERR_CUDA, "reading the device state failed");
            }
            ok = fwrite(buf.data(), 1, len, fp) == len;
        }
        if (fclose(fp) != 0) ok = false;
        if (!ok) return fail(PIC_ERR_ARG, "writing %s failed", path);
        return PIC_OK;
    }

    int load(const char *path) {
        FILE *fp = fopen(path, "rb");
        if (!fp) return fail(PIC_ERR_ARG, "cannot open %s", path);
        auto reject = [&](const char *why) {
            fclose(fp);
            return fail(PIC_ERR_ARG, "checkpoint %s: %s", path, why);
        };
        SaveHeader hd{};
        if (fread(&hd, sizeof hd, 1, fp) != 1 || memcmp(hd.magic, "PICSAVE1", 8) != 0 || hd.version != 2)
            return reject("not a checkpoint of this library version");
        bool same = hd.precision == cfg.precision && hd.arena_bytes == arena_bytes &&
                    hd.max_particles == cfg.max_particles && hd.max_probes == cfg.max_probes &&
                    hd.max_freqs == cfg.max_freqs && hd.dt == cfg.dt && hd.eps0 == cfg.eps0 && hd.mu0 == cfg.mu0 &&
                    hd.cpml_cells == cfg.cpml_cells && hd.cpml_order == cfg.cpml_order &&
                    hd.cpml_sigma_fac == cfg.cpml_sigma_fac && hd.cpml_kappa_max == cfg.cpml_kappa_max &&
                    hd.cpml_alpha_max == cfg.cpml_alpha_max && hd.flags == cfg.flags &&
                    (hd.fused_ready == 0 || (hd.fused_ready == 1 && fused));
        for (int a = 0; a < 3; a++) same = same && hd.n[a] == n[a] && hd.d[a] == d[a];
        for (int q6 = 0; q6 < 6; q6++) same = same && hd.bc[q6] == cfg.bc[q6];
        if (!same) return reject("written by a differently configured simulation");
        // counters: everything a kernel indexes with must lie inside this handle's capacities
        if (hd.np < 0 || hd.np > cfg.max_particles || hd.probe_np < 0 || hd.probe_np > cfg.max_probes ||
            hd.probe_nf < 0 || hd.probe_nf > cfg.max_freqs || (hd.probe_mask & ~7u) || hd.buffered < 0 ||
            hd.buffered >= DFT_BLOCK || hd.since_sort < 1 || hd.since_sort > DFT_BLOCK || hd.step_host < 0 ||
            hd.nsources < 0 || hd.nsources > MAX_SOURCES || (hd.bold_stale & ~1) || (hd.have_q & ~1) ||
            (hd.deposit & ~1) || (hd.have_q && !(std::isfinite(hd.q) && std::isfinite(hd.m) && hd.m > 0.0)))
            return reject("counters outside this handle's capacities");
        std::vector<Source> src((size_t)hd.nsources);
        if (hd.nsources && fread(src.data(), sizeof(Source), src.size(), fp) != src.size())
            return reject("truncated");
        for (const Source &sr : src) {
            bool ok = sr.comp >= 0 && sr.comp < 3;
            for (int a = 0; a < 3; a++)
                ok = ok && sr.box[2 * a] >= 0 && sr.box[2 * a] <= sr.box[2 * a + 1] && sr.box[2 * a + 1] <= n[a];
            if (!ok) return reject("a source outside the grid");
        }
        // the whole arena must be there before anything is copied
        const long body = ftell(fp);
        if (body < 0 || fseek(fp, 0, SEEK_END) != 0) return reject("cannot be sized");
        const long total = ftell(fp);
        if (total < 0 || (unsigned long)total != (unsigned long)body + arena_bytes) return reject("truncated or too long");
        int rc = sync();
        if (rc) { fclose(fp); return rc; }
        // the configuration's own arrays must match this handle's byte for byte
        for (const auto &reg : config_regions()) {
            std::vector<char> a(reg.second), b(reg.second);
            if (fseek(fp, body + (long)reg.first, SEEK_SET) != 0 || fread(a.data(), 1, a.size(), fp) != a.size())
                return reject("truncated");
            if (cudaMemcpy(b.data(), (char *)arena + reg.first, b.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
                fclose(fp);
                return fail(PIC_ERR_CUDA, "reading the device state failed");
            }
            if (memcmp(a.data(), b.data(), a.size()) != 0)
                return reject("materials or absorbing layers differ from this handle's configuration");
        }
        if (fseek(fp, body, SEEK_SET) != 0) return reject("cannot be read");
        std::vector<char> buf;
        const size_t chunk = (size_t)64 << 20;
        for (size_t off = 0; off < arena_bytes; off += chunk) {
            const size_t len = std::min(chunk, arena_bytes - off);
            buf.resize(len);
            if (fread(buf.data(), 1, len, fp) != len) {
                fclose(fp);
                return fail(PIC_ERR_ARG, "truncated checkpoint %s", path);
            }
            if (cudaMemcpy((char *)arena + off, buf.data(), len, cudaMemcpyHostToDevice) != cudaSuccess) {
                fclose(fp);
                return fail(PIC_ERR_CUDA, "writing the device state failed");
            }
        }
        fclose(fp);
        drop_graph();
        fused_ready = hd.fused_ready != 0;
        sources = src;
        step_host = hd.step_host;
        p.n = hd.np;
        buffered = hd.buffered;
        since_sort = hd.since_sort;
        bold_stale = hd.bold_stale != 0;
        have_q = hd.have_q != 0;
        q = hd.q;
        m = hd.m;
        pp.deposit = hd.deposit;
        pr.np = hd.probe_np;
        pr.nf = hd.probe_nf;
        pr.mask = hd.probe_mask;
        if (have_q) {
            pp.qmdt2 = (T)(q * cfg.dt / (2.0 * m));
            for (int c = 0; c < 3; c++) {
                const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
                pp.jscale[c] = (T)(-q / (cfg.dt * d[a1] * d[a2]));
            }
        }
        return PIC_OK;
    }

    // ---------------------------------------------------------- tuning --
    pic_tuning tuning() const { return pic_tuning{pp.dep_smem, sort_every, fplan.block, (fused && use_fused) ? 1 : 0}; }
    int set_tuning(const pic_tuning &t) override {
        const int dep = t.dep_smem_bytes, every = t.sort_every, blk = t.field_block;
        if (t.field_path != 0 && t.field_path != 1) return fail(PIC_ERR_ARG, "field_path %d is not 0 or 1", t.field_path);
        if (dep < 0 || dep > DEP_SMEM_MAX || dep % 16 != 0)
            return fail(PIC_ERR_ARG, "dep_smem_bytes %d outside 0..%d or not a multiple of 16", dep, DEP_SMEM_MAX);
        if (every < 1 || every > DFT_BLOCK || DFT_BLOCK % every != 0)
            return fail(PIC_ERR_ARG, "sort_every %d does not divide %d", every, DFT_BLOCK);
        if (blk != 128 && blk != 256 && blk != 512)
            return fail(PIC_ERR_ARG, "field_block %d is not 128, 256 or 512", blk);
        const bool uf = t.field_path == 1;
        if (uf != use_fused) {  // switch the field path (the state moves back to f when leaving the fused one)
            if (!uf) {
                int rc = leave_fused();
                if (rc) return rc;
            }
            use_fused = uf;
            drop_graph();
        }
        if (dep != pp.dep_smem || every != sort_every || blk != fplan.block) {
            pp.dep_smem = dep;
            sort_every = every;
            fplan.block = blk;
            drop_graph();  // the captured launches hold the old settings
        }
        return PIC_OK;
    }

    // one whole block under the current tuning, timed on the stream (the
    // graph is captured before the start event)
    int time_block(cudaEvent_t e0, cudaEvent_t e1, double *us) {
        int rc = prepare();
        if (rc) return rc;
        rc = ensure_graph();
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(e0, stream));
        rc = step(DFT_BLOCK);
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(e1, stream));
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        *us = 1e3 * ms / DFT_BLOCK;
        return PIC_OK;
    }

    int tune(int rounds, pic_tune_report *rep) {
        if (rounds < 1 || rounds > 16) return fail(PIC_ERR_ARG, "rounds must be 1..16");
        const long long s0 = step_host;
        int rc = PIC_OK;
        if (buffered) rc = step(DFT_BLOCK - buffered);  // reach a block boundary
        if (rc) return rc;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        {
            cudaError_t ce = cudaEventCreate(&e0);
            if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
            if (ce != cudaSuccess) {
                if (e0) cudaEventDestroy(e0);
                return fail(PIC_ERR_CUDA, "tuning events: %s", cudaGetErrorString(ce));
            }
        }
        const int deps[5] = {0, 2048, 4096, 8192, 16384}, everies[4] = {8, 16, 32, 64}, blocks[3] = {128, 256, 512};
        pic_tuning cand[PIC_TUNE_MAX_CANDIDATES];
        double best_us[PIC_TUNE_MAX_CANDIDATES];
        int nc = 0;
        // time candidates [first, first + count) `rounds` times each; *win = the fastest
        auto pass = [&](int first, int count, int *win) -> int {
            for (int r = 0; r < rounds; r++)
                for (int c = first; c < first + count; c++) {
                    int q = set_tuning(cand[c]);
                    if (q) return q;
                    double us = 0.0;
                    q = time_block(e0, e1, &us);
                    if (q) return q;
                    best_us[c] = std::min(best_us[c], us);
                }
            *win = first;
            for (int c = first; c < first + count; c++)
                if (best_us[c] < best_us[*win]) *win = c;
            return PIC_OK;
        };
        const pic_tuning t0 = tuning();
        for (int d : deps) { cand[nc] = pic_tuning{d, t0.sort_every, t0.field_block, t0.field_path}; best_us[nc++] = 1e300; }
        int win = 0;
        rc = pass(0, 5, &win);
        if (!rc) {
            const pic_tuning t = cand[win];
            for (int e : everies) { cand[nc] = pic_tuning{t.dep_smem_bytes, e, t.field_block, t.field_path}; best_us[nc++] = 1e300; }
            rc = pass(5, 4, &win);
        }
        if (!rc) {
            const pic_tuning t = cand[win];
            for (int b : blocks) { cand[nc] = pic_tuning{t.dep_smem_bytes, t.sort_every, b, t.field_path}; best_us[nc++] = 1e300; }
            rc = pass(9, 3, &win);
        }
        if (!rc && fused) {  // the fused pass against the split updates
            const pic_tuning t = cand[win];
            for (int fp : {1, 0}) { cand[nc] = pic_tuning{t.dep_smem_bytes, t.sort_every, t.field_block, fp}; best_us[nc++] = 1e300; }
            rc = pass(12, 2, &win);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        const pic_tuning best = cand[win];
        rc = set_tuning(best);
        if (rc) return rc;
        if (rep) {
            std::memset(rep, 0, sizeof(*rep));
            rep->best = best;
            rep->n = nc;
            rep->best_lanes = -1;
            for (int c = 0; c < nc; c++) {
                rep->cand[c] = cand[c];
                rep->us_per_step[c] = best_us[c];
                rep->lanes[c] = -1;
            }
            rep->steps = step_host - s0;
        }
        return sync();
    }

    int profile_steps(long long nsteps, double *out) {
        int rc = prepare();
        if (rc) return rc;
        for (int q6 = 0; q6 < 6; q6++) out[q6] = 0.0;
        if (nsteps <= 0) return PIC_OK;
        // The steps run exactly as pic_step runs them (same streams and
        // overlap), with timing events at the phase boundaries.
        constexpr int NE = 9;
        const int B = DFT_BLOCK;
        std::vector<cudaEvent_t> ev((size_t)B * NE);
        for (auto &e : ev) CUDA_TRY(cudaEventCreate(&e));
        long long done = 0;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        while (done < nsteps) {
            const int cnt = (int)std::min<long long>(B, nsteps - done);
            for (int s = 0; s < cnt; s++) {
                cudaEvent_t *e = &ev[(size_t)s * NE];
                const bool sort = since_sort >= sort_every;
                launch_step(sort, true, e, (int)(step_host & 1));
                since_sort = sort ? 1 : since_sort + 1;
                buffered++;
                step_host++;
                if (buffered == DFT_BLOCK) {
                    launch_dft_flush<T>(pr, d_step, DFT_BLOCK, stream);
                    buffered = 0;
                }
                cudaEventRecord(e[7], stream);
            }
            CUDA_TRY(cudaGetLastError());
            CUDA_TRY(cudaEventSynchronize(ev[(size_t)(cnt - 1) * NE + 7]));
            for (int s = 0; s < cnt; s++) {
                cudaEvent_t *e = &ev[(size_t)s * NE];
                // fused path: the pass runs from its start (8) to 1, beside the push (2 to 3)
                const int f0 = fused_ready ? 8 : 0;
                const int from[6] = {f0, 2, 4, 5, 6, 0}, to[6] = {1, 3, 5, 6, 7, 7};
                for (int q6 = 0; q6 < 6; q6++) {
                    float ms;
                    cudaEventElapsedTime(&ms, e[from[q6]], e[to[q6]]);
                    acc[q6] += ms;
                }
            }
            done += cnt;
        }
        for (auto &e : ev) cudaEventDestroy(e);
        for (int q6 = 0; q6 < 6; q6++) out[q6] = acc[q6] * 1000.0 / (double)nsteps;
        return sync();
    }
};

struct pic_handle {
    int precision;
    SimBase *sim;
};

template <typename T>
static Sim<T> *S(pic_handle *h) {
    return static_cast<Sim<T> *>(h->sim);
}

#define DISPATCH(h, call)                                                       \
    ((h)->precision == PIC_FP64 ? S<double>(h)->call : S<float>(h)->call)

// ---------------------------------------------------------- entry points --
template <typename T>
static int add_particles_t(Sim<T> *s, int64_t n, const double *xyz, const double *u, double q, double m,
                           int64_t *n_rejected) {
    if (n_rejected) *n_rejected = 0;
    if (n < 0 || (n > 0 && (!xyz || !u))) return fail(PIC_ERR_ARG, "bad particle arrays");
    if (!(m > 0.0) || !std::isfinite(q)) return fail(PIC_ERR_ARG, "need m_macro > 0 and finite q_macro");
    if (s->have_q && (q != s->q || m != s->m)) return fail(PIC_ERR_ARG, "all particles must share q_macro and m_macro");
    if (s->p.n + n > s->cfg.max_particles)
        return fail(PIC_ERR_OOM, "%lld particles exceed max_particles=%lld", (long long)(s->p.n + n),
                    (long long)s->cfg.max_particles);
    // One kernel converts the caller's arrays into the particle arrays beyond
    // the live count and counts the electrons outside the allowed region and
    // those inside a metal.  It reads the arrays where they are on a device
    // with coherent access to pageable host memory, else from copies in the
    // sort's scratch arrays (free between steps).
    const long long base = s->p.n;
    if (n > 0) {
        const size_t bytes = (size_t)n * 3 * sizeof(double);
        char *stage = reinterpret_cast<char *>(s->psort.cell[0]);
        const size_t room = (size_t)(reinterpret_cast<char *>(s->psort.id + s->cfg.max_particles) - stage);
        if (2 * bytes + 16 > room) return fail(PIC_ERR_OOM, "particle staging area too small");
        const double *d_xyz = reinterpret_cast<double *>(stage);
        const double *d_u = reinterpret_cast<double *>(stage + (bytes + 15) / 16 * 16);
        unsigned long long *d_cnt = reinterpret_cast<unsigned long long *>(s->d_keyset);  // scratch after create
        CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 2 * sizeof(unsigned long long), s->stream));
        if (s->host_direct) {  // the kernel reads the caller's arrays where they are (synchronised below)
            d_xyz = xyz;
            d_u = u;
        } else {
            CUDA_TRY(cudaMemcpyAsync(const_cast<double *>(d_xyz), xyz, bytes, cudaMemcpyHostToDevice, s->stream));
            CUDA_TRY(cudaMemcpyAsync(const_cast<double *>(d_u), u, bytes, cudaMemcpyHostToDevice, s->stream));
        }
        ParticleIn in{};
        for (int a = 0; a < 3; a++) {
            in.d[a] = s->d[a];
            in.n[a] = s->n[a];
            in.per[a] = s->g.per[a];
        }
        launch_particles_in<T>(d_xyz, d_u, n, base, in, s->p, s->d_mat, s->d_mat_metal, d_cnt, s->stream);
        CUDA_TRY(cudaGetLastError());
        unsigned long long cnt[2] = {0, 0};
        CUDA_TRY(cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (cnt[0]) {
            if (n_rejected) *n_rejected = (int64_t)cnt[0];
            return fail(PIC_ERR_ARG, "%lld particles outside the allowed region", (long long)cnt[0]);
        }
        if (cnt[1]) {
            if (n_rejected) *n_rejected = (int64_t)cnt[1];
            return fail(PIC_ERR_ARG, "%lld particles inside a metal cell", (long long)cnt[1]);
        }
    }
    s->p.n = base + n;
    s->have_q = true;
    s->q = q;
    s->m = m;
    s->pp.qmdt2 = (T)(q * s->cfg.dt / (2.0 * m));
    for (int c = 0; c < 3; c++) {
        const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
        s->pp.jscale[c] = (T)(-q / (s->cfg.dt * s->d[a1] * s->d[a2]));
    }
    s->bold_stale = true;
    s->since_sort = DFT_BLOCK;  // the new electrons are in input order: sort before the next push
    s->drop_graph();
    return PIC_OK;
}

template <typename T>
static int get_particles_t(Sim<T> *s, double *xyz, double *u, uint8_t *status) {
    int rc = s->sync();
    if (rc) return rc;
    const long long n = s->p.n;
    std::vector<int> cell[3];
    std::vector<T> off[3], uu[3], ul[3];
    std::vector<uint8_t> st(n);
    std::vector<long long> id(n);
    for (int a = 0; a < 3; a++) {
        cell[a].resize(n); off[a].resize(n); uu[a].resize(n); ul[a].resize(n);
        CUDA_TRY(cudaMemcpy(ul[a].data(), s->p.ulo[a], n * sizeof(T), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(cell[a].data(), s->p.cell[a], n * sizeof(int), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(off[a].data(), s->p.off[a], n * sizeof(T), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(uu[a].data(), s->p.u[a], n * sizeof(T), cudaMemcpyDeviceToHost));
    }
    CUDA_TRY(cudaMemcpy(st.data(), s->p.status, n, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(id.data(), s->p.id, n * sizeof(long long), cudaMemcpyDeviceToHost));
    for (long long q2 = 0; q2 < n; q2++) {
        const long long o = id[q2];
        if (o < 0 || o >= n) return fail(PIC_ERR_DEVICE, "corrupt particle id");
        for (int a = 0; a < 3; a++) {
            if (xyz) xyz[3 * o + a] = ((double)cell[a][q2] + (double)off[a][q2]) * s->d[a];
            if (u) u[3 * o + a] = (double)uu[a][q2] + (double)ul[a][q2];
        }
        if (status) status[o] = st[q2];
    }
    return PIC_OK;
}

template <typename T>
static int probe_dft_t(Sim<T> *s, int np, const double *xyz, uint32_t mask, int nf, const double *freq) {
    if (np < 0 || nf < 0 || (mask & ~7u)) return fail(PIC_ERR_ARG, "bad probe arguments");
    if (np > s->cfg.max_probes || nf > s->cfg.max_freqs)
        return fail(PIC_ERR_OOM, "probe capacity is %d x %d", s->cfg.max_probes, s->cfg.max_freqs);
    if ((np > 0 && !xyz) || (nf > 0 && !freq)) return fail(PIC_ERR_ARG, "NULL probe arrays");
    std::vector<double> cells((size_t)np * 3);
    for (int q2 = 0; q2 < np; q2++)
        for (int a = 0; a < 3; a++) {
            double xi = xyz[3 * q2 + a] / s->d[a];
            if (!std::isfinite(xi)) return fail(PIC_ERR_ARG, "non-finite probe position");
            if (!s->g.per[a] && (xi < 1.0 || xi >= s->n[a] - 1.0))
                return fail(PIC_ERR_ARG, "probe %d lies within one cell of a face", q2);
            cells[3 * q2 + a] = xi;
        }
    // interpolation stencil of every (probe, component): 8 corners of the
    // component's staggered lattice, index and trilinear weight
    std::vector<long long> st_idx((size_t)np * 24);
    std::vector<T> st_w((size_t)np * 24);
    for (int q2 = 0; q2 < np; q2++)
        for (int c = 0; c < 3; c++)
            for (int corner = 0; corner < 8; corner++) {
                long long idx = 0, stride = 1;
                double wt = 1.0;
                for (int a = 0; a < 3; a++) {
                    const double sa = cells[3 * q2 + a] - (a == c ? 0.5 : 0.0);
                    const double fl = std::floor(sa);
                    const int bit = (corner >> a) & 1;
                    int ib = (int)fl + bit;
                    const int na = s->n[a];
                    if (s->g.per[a]) ib = ((ib % na) + na) % na;
                    else ib = std::min(std::max(ib, 0), na - 1);
                    wt *= bit ? (sa - fl) : 1.0 - (sa - fl);
                    idx += (long long)ib * stride;
                    stride *= na;
                }
                st_idx[(size_t)q2 * 24 + c * 8 + corner] = idx;
                st_w[(size_t)q2 * 24 + c * 8 + corner] = (T)wt;
            }
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (np) CUDA_TRY(cudaMemcpy(s->d_probe_xyz, cells.data(), cells.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (np) CUDA_TRY(cudaMemcpy(s->d_st_idx, st_idx.data(), st_idx.size() * sizeof(long long), cudaMemcpyHostToDevice));
    if (np) CUDA_TRY(cudaMemcpy(s->d_st_w, st_w.data(), st_w.size() * sizeof(T), cudaMemcpyHostToDevice));
    if (nf) CUDA_TRY(cudaMemcpy(s->d_freq, freq, nf * sizeof(double), cudaMemcpyHostToDevice));
    if (np && nf) CUDA_TRY(cudaMemset(s->d_F, 0, (size_t)np * 3 * nf * 2 * sizeof(double)));
    s->pr.np = np;
    s->pr.nf = nf;
    s->pr.mask = mask;
    s->buffered = 0;
    s->drop_graph();
    return PIC_OK;
}

template <typename T>
static int probe_read_t(Sim<T> *s, double *out) {
    if (s->pr.np == 0 || s->pr.nf == 0) return fail(PIC_ERR_STATE, "no probes configured");
    int rc = s->flush_probes();
    if (rc) return rc;
    rc = s->sync();
    if (rc) return rc;
    CUDA_TRY(cudaMemcpy(out, s->d_F, (size_t)s->pr.np * 3 * s->pr.nf * 2 * sizeof(double), cudaMemcpyDeviceToHost));
    return PIC_OK;
}

template <typename T>
static int probe_kw_t(Sim<T> *s, int comp, int axis, int nk, const double *k, double *out) {
    if (s->pr.np == 0 || s->pr.nf == 0) return fail(PIC_ERR_STATE, "no probes configured");
    if (comp < 0 || comp > 2 || axis < 0 || axis > 2 || nk < 0 || (nk > 0 && (!k || !out)))
        return fail(PIC_ERR_ARG, "bad k-omega arguments");
    if (nk > 65535) return fail(PIC_ERR_ARG, "at most 65535 wavenumbers");
    if (nk == 0) return PIC_OK;
    int rc = s->flush_probes();
    if (rc) return rc;
    const size_t kb = (size_t)nk * sizeof(double), ob = (size_t)nk * s->pr.nf * sizeof(double);
    double *dk = nullptr, *dout = nullptr;
    CUDA_TRY(cudaMalloc(&dk, kb));
    if (cudaMalloc(&dout, ob) != cudaSuccess) {
        cudaFree(dk);
        return fail(PIC_ERR_OOM, "k-omega output of %zu bytes", ob);
    }
    cudaError_t e = cudaMemcpyAsync(dk, k, kb, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) {
        launch_probe_kw(s->d_F, s->d_probe_xyz, s->d[axis], axis, s->pr.np, s->pr.nf, comp, dk, nk, dout, s->stream);
        s->kernels += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, ob, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(dk);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(PIC_ERR_CUDA, "k-omega map: %s", cudaGetErrorString(e));
    return s->sync();
}

template <typename T>
static T *field_of(Sim<T> *s, int which) {
    const int c = which % 3;
    const Fields<T> v = s->current();
    switch (which / 3) {
    case 0: return v.E[c];
    case 1: return v.H[c];
    case 2: return v.Jp[c];
    default: return v.Jf[c];
    }
}

template <typename T>
static int get_field_t(Sim<T> *s, int which, double *out) {
    if (which < 0 || which > 11 || !out) return fail(PIC_ERR_ARG, "bad field id");
    int rc = s->sync();
    if (rc) return rc;
    std::vector<T> tmp((size_t)s->N);
    CUDA_TRY(cudaMemcpy(tmp.data(), field_of(s, which), (size_t)s->N * sizeof(T), cudaMemcpyDeviceToHost));
    for (size_t e = 0; e < (size_t)s->N; e++) out[e] = (double)tmp[e];
    return PIC_OK;
}

template <typename T>
static int set_field_t(Sim<T> *s, int which, const double *in) {
    if (which < 0 || which > 5 || !in) return fail(PIC_ERR_ARG, "only E and H components can be set");
    int rc = s->sync();
    if (rc) return rc;
    rc = s->leave_fused();  // back to the plain state: the next step starts the fused path again
    if (rc) return rc;
    std::vector<T> tmp((size_t)s->N);
    for (size_t e = 0; e < (size_t)s->N; e++) tmp[e] = (T)in[e];
    CUDA_TRY(cudaMemcpy(field_of(s, which), tmp.data(), (size_t)s->N * sizeof(T), cudaMemcpyHostToDevice));
    if (which >= PIC_HX) s->bold_stale = true;
    return PIC_OK;
}

template <typename T>
static int stats_t(Sim<T> *s, pic_stats *out) {
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return fail(PIC_ERR_CUDA, "%s", cudaGetErrorString(e));
    pic::launch_nonfinite_scan<T>(s->current(), s->N, s->d_err, s->stream);
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    int err = 0;
    CUDA_TRY(cudaMemcpy(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<uint8_t> st((size_t)s->p.n);
    if (s->p.n) CUDA_TRY(cudaMemcpy(st.data(), s->p.status, (size_t)s->p.n, cudaMemcpyDeviceToHost));
    long long fr = 0;
    for (auto v : st) fr += v != 0;
    out->step = s->step_host;
    out->n_particles = s->p.n;
    out->n_frozen = fr;
    out->device_error = err;
    out->n_edge_classes = s->n_classes;
    out->kernel_launches = s->kernels;
    out->field_path = (s->fused && s->use_fused) ? 1 : 0;
    return PIC_OK;
}

extern "C" {

const char *pic_last_error(void) { return g_err.c_str(); }

int pic_workspace_size(const pic_config *cfg, size_t *bytes) {
    g_err.clear();
    int rc = validate(cfg);
    if (rc) return rc;
    if (!bytes) return fail(PIC_ERR_ARG, "bytes is NULL");
    Arena a;
    if (cfg->precision == PIC_FP64) {
        Sim<double> s;
        s.init_geometry(cfg);
        s.plan(a);
    } else {
        Sim<float> s;
        s.init_geometry(cfg);
        s.plan(a);
    }
    *bytes = a.used;
    return PIC_OK;
}

int pic_create(const pic_config *cfg, pic_handle **out) {
    NvtxRange nvtx_range("pic_create");
    g_err.clear();
    if (!out) return fail(PIC_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = validate(cfg);
    if (rc) return rc;
    pic_handle *h = new pic_handle;
    h->precision = cfg->precision;
    if (cfg->precision == PIC_FP64) {
        auto *s = new Sim<double>;
        h->sim = s;
        rc = s->create(cfg);
    } else {
        auto *s = new Sim<float>;
        h->sim = s;
        rc = s->create(cfg);
    }
    if (rc) {
        std::string msg = g_err;
        delete h->sim;
        delete h;
        g_err = msg;
        return rc;
    }
    *out = h;
    return PIC_OK;
}

int pic_destroy(pic_handle *h) {
    NvtxRange nvtx_range("pic_destroy");
    g_err.clear();
    if (!h) return PIC_OK;
    delete h->sim;
    delete h;
    return PIC_OK;
}

int pic_set_stream(pic_handle *h, void *stream) {
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    auto apply = [&](auto *s) -> int {
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        s->drop_graph();
        if (s->own_stream) { cudaStreamDestroy(s->stream); s->own_stream = false; }
        if (stream) {
            s->stream = (cudaStream_t)stream;
        } else {
            CUDA_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
            s->own_stream = true;
        }
        return PIC_OK;
    };
    return h->precision == PIC_FP64 ? apply(S<double>(h)) : apply(S<float>(h));
}

int pic_add_particles(pic_handle *h, int64_t n, const double *xyz, const double *u, double q_macro,
                      double m_macro, int64_t *n_rejected) {
    NvtxRange nvtx_range("pic_add_particles");
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    return h->precision == PIC_FP64 ? add_particles_t(S<double>(h), n, xyz, u, q_macro, m_macro, n_rejected)
                                    : add_particles_t(S<float>(h), n, xyz, u, q_macro, m_macro, n_rejected);
}

int pic_get_particles(pic_handle *h, double *xyz, double *u, uint8_t *status) {
    NvtxRange nvtx_range("pic_get_particles");
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    return h->precision == PIC_FP64 ? get_particles_t(S<double>(h), xyz, u, status)
                                    : get_particles_t(S<float>(h), xyz, u, status);
}

int pic_set_deposit(pic_handle *h, int on) {
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    if (h->precision == PIC_FP64) { S<double>(h)->pp.deposit = on != 0; S<double>(h)->drop_graph(); }
    else { S<float>(h)->pp.deposit = on != 0; S<float>(h)->drop_graph(); }
    return PIC_OK;
}

int pic_add_source(pic_handle *h, int comp, const int64_t *box, double amp, double t0, double tau, double f0) {
    g_err.clear();
    if (!h || !box) return fail(PIC_ERR_ARG, "NULL argument");
    if (comp < 0 || comp > 2 || !(tau > 0.0) || f0 < 0.0) return fail(PIC_ERR_ARG, "bad source parameters");
    auto apply = [&](auto *s) -> int {
        if ((int)s->sources.size() >= MAX_SOURCES) return fail(PIC_ERR_ARG, "at most %d sources", MAX_SOURCES);
        Source src{};
        src.comp = comp;
        for (int a = 0; a < 3; a++) {
            if (box[2 * a] < 0 || box[2 * a + 1] > s->n[a] || box[2 * a] >= box[2 * a + 1])
                return fail(PIC_ERR_ARG, "source box outside the grid on axis %d", a);
            src.box[2 * a] = (int)box[2 * a];
            src.box[2 * a + 1] = (int)box[2 * a + 1];
        }
        src.amp = amp; src.t0 = t0; src.tau = tau; src.f0 = f0;
        s->sources.push_back(src);
        s->drop_graph();
        return PIC_OK;
    };
    return h->precision == PIC_FP64 ? apply(S<double>(h)) : apply(S<float>(h));
}

int pic_probe_dft(pic_handle *h, int np, const double *xyz, uint32_t comp_mask, int nf, const double *freq_hz) {
    NvtxRange nvtx_range("pic_probe_dft");
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    return h->precision == PIC_FP64 ? probe_dft_t(S<double>(h), np, xyz, comp_mask, nf, freq_hz)
                                    : probe_dft_t(S<float>(h), np, xyz, comp_mask, nf, freq_hz);
}

int pic_step(pic_handle *h, int64_t nsteps) {
    NvtxRange nvtx_range("pic_step");
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    return DISPATCH(h, step(nsteps));
}

int pic_sync(pic_handle *h) {
    NvtxRange nvtx_range("pic_sync");
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    return DISPATCH(h, check());
}

int pic_probe_read(pic_handle *h, double *out) {
    NvtxRange nvtx_range("pic_probe_read");
    g_err.clear();
    if (!h || !out) return fail(PIC_ERR_ARG, "NULL argument");
    return h->precision == PIC_FP64 ? probe_read_t(S<double>(h), out) : probe_read_t(S<float>(h), out);
}

int pic_probe_kw(pic_handle *h, int comp, int axis, int nk, const double *k, double *out) {
    NvtxRange nvtx_range("pic_probe_kw");
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    return h->precision == PIC_FP64 ? probe_kw_t(S<double>(h), comp, axis, nk, k, out)
                                    : probe_kw_t(S<float>(h), comp, axis, nk, k, out);
}

int pic_get_field(pic_handle *h, int which, double *out) {
    NvtxRange nvtx_range("pic_get_field");
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    return h->precision == PIC_FP64 ? get_field_t(S<double>(h), which, out) : get_field_t(S<float>(h), which, out);
}

int pic_set_field(pic_handle *h, int which, const double *in) {
    NvtxRange nvtx_range("pic_set_field");
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    return h->precision == PIC_FP64 ? set_field_t(S<double>(h), which, in) : set_field_t(S<float>(h), which, in);
}

int pic_get_stats(pic_handle *h, pic_stats *out) {
    g_err.clear();
    if (!h || !out) return fail(PIC_ERR_ARG, "NULL argument");
    return h->precision == PIC_FP64 ? stats_t(S<double>(h), out) : stats_t(S<float>(h), out);
}

int pic_save(pic_handle *h, const char *path) {
    NvtxRange nvtx_range("pic_save");
    g_err.clear();
    if (!h || !path) return fail(PIC_ERR_ARG, "NULL argument");
    return DISPATCH(h, save(path));
}

int pic_load(pic_handle *h, const char *path) {
    NvtxRange nvtx_range("pic_load");
    g_err.clear();
    if (!h || !path) return fail(PIC_ERR_ARG, "NULL argument");
    return DISPATCH(h, load(path));
}

int pic_profile_steps(pic_handle *h, int64_t nsteps, double *out_us) {
    NvtxRange nvtx_range("pic_profile_steps");
    g_err.clear();
    if (!h || !out_us) return fail(PIC_ERR_ARG, "NULL argument");
    return DISPATCH(h, profile_steps(nsteps, out_us));
}

int pic_get_tuning(pic_handle *h, pic_tuning *out) {
    g_err.clear();
    if (!h || !out) return fail(PIC_ERR_ARG, "NULL argument");
    *out = h->precision == PIC_FP64 ? S<double>(h)->tuning() : S<float>(h)->tuning();
    return PIC_OK;
}

int pic_set_tuning(pic_handle *h, const pic_tuning *t) {
    g_err.clear();
    if (!h || !t) return fail(PIC_ERR_ARG, "NULL argument");
    return DISPATCH(h, set_tuning(*t));
}

int pic_tune(pic_handle *h, int32_t rounds, pic_tune_report *report) {
    NvtxRange nvtx_range("pic_tune");
    g_err.clear();
    if (!h) return fail(PIC_ERR_ARG, "NULL handle");
    return DISPATCH(h, tune(rounds, report));
}

}  // extern "C"

// ------------------------------------------------------------------ batch --
// Several independent simulations stepped together: whole DFT_BLOCK-step
// blocks of every instance are captured into one CUDA graph (one branch per
// instance, each on its own streams), so small grids share the GPU instead
// of running one after another.
struct pic_batch {
    std::vector<pic_handle *> h;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> epochs, kernels;
    int lanes = 0;  // instances that run side by side; 0: all of them
    bool joint = true;  // the fused passes of the instances that take one run as one joint pass per step
    int joint_chunk = 32;  // planes per work item of the joint pass (0: each instance's own)
    cudaStream_t jaux[3] = {nullptr, nullptr, nullptr};  // slab kinds of the joint pass
    FusedInst *d_tab = nullptr;
    int4 *d_items = nullptr;
    size_t tab_cap = 0, items_cap = 0;

    void drop() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    bool stale() const {
        if (!exec) return true;
        for (size_t i = 0; i < h.size(); i++)
            if (h[i]->sim->graph_epoch() != epochs[i]) return true;
        return false;
    }
    // The joint pass's tables for the instances J (before the capture; the
    // previous batch graph may still read the old ones).
    int joint_tables(const std::vector<int> &J, FusedJoint &jt) {
        std::vector<FusedInst> tab(J.size());
        std::vector<int4> items[4];
        for (size_t q = 0; q < J.size(); q++) {
            const int chunk = joint_chunk > 0 ? joint_chunk : h[J[q]]->sim->fused_chunk_planes();
            h[J[q]]->sim->joint_entry(tab[q], chunk);
            h[J[q]]->sim->joint_items((int)q, chunk, items);
        }
        size_t nitems = 0;
        for (auto &v : items) nitems += v.size();
        CUDA_TRY(cudaStreamSynchronize(stream));
        if (tab.size() > tab_cap) {
            if (d_tab) cudaFree(d_tab);
            d_tab = nullptr;
            tab_cap = 0;
            CUDA_TRY(cudaMalloc(&d_tab, tab.size() * sizeof(FusedInst)));
            tab_cap = tab.size();
        }
        if (nitems > items_cap) {
            if (d_items) cudaFree(d_items);
            d_items = nullptr;
            items_cap = 0;
            CUDA_TRY(cudaMalloc(&d_items, nitems * sizeof(int4)));
            items_cap = nitems;
        }
        CUDA_TRY(cudaMemcpy(d_tab, tab.data(), tab.size() * sizeof(FusedInst), cudaMemcpyHostToDevice));
        size_t off = 0;
        jt = FusedJoint{};
        jt.tab = d_tab;
        for (int k = 0; k < 4; k++) {
            if (!items[k].empty())
                CUDA_TRY(cudaMemcpy(d_items + off, items[k].data(), items[k].size() * sizeof(int4),
                                    cudaMemcpyHostToDevice));
            jt.items[k] = d_items + off;
            jt.nitems[k] = (int)items[k].size();
            off += items[k].size();
        }
        return PIC_OK;
    }
    int capture() {
        drop();
        // Instances whose fused pass joins the joint pass (J, two or more)
        // and the others (R), which run whole blocks of their own.
        std::vector<int> J, R;
        for (size_t i = 0; i < h.size(); i++) (joint && h[i]->sim->joint_capable() ? J : R).push_back((int)i);
        if (J.size() < 2) {
            R.insert(R.end(), J.begin(), J.end());
            J.clear();
        }
        FusedJoint jt{};
        if (!J.empty()) {
            const int rc = joint_tables(J, jt);
            if (rc) return rc;
        }
        const long long count0 = launch_count();
        CUDA_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        // The instances of R are dealt to `lanes` chains (largest first, each
        // to the chain with the fewest cells so far); the chains fork from the
        // start of the capture, and within a chain each instance's block starts
        // when the one before it has finished.  One chain per instance: every
        // instance runs beside every other.
        const int nl = (lanes <= 0 || lanes >= (int)R.size()) ? (int)R.size() : lanes;
        std::vector<int> order(R);
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return h[a]->sim->cells() > h[b]->sim->cells(); });
        std::vector<long long> load(nl, 0);
        std::vector<cudaStream_t> tail(nl, stream);
        for (int i : order) {
            const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            kernels[i] = h[i]->sim->launch_block_on(tail[l]);
            tail[l] = h[i]->sim->main_stream();
            load[l] += h[i]->sim->cells();
        }
        // The instances of J step together: per step, each one's sort, push
        // and sources on its own streams beside one joint pass over all of
        // them (the pass reads only what those leave alone), then each one's
        // correction and probe sample after both.
        for (int i : J) kernels[i] = 0;
        for (int st = 0; st < DFT_BLOCK && !J.empty(); st++) {
            for (int i : J) kernels[i] += h[i]->sim->joint_pre(st, stream);
            jt.phase = st & 1;
            cudaEventRecord(ev, stream);
            for (cudaStream_t x : jaux) cudaStreamWaitEvent(x, ev, 0);
            const long long k0 = launch_count();
            launch_fused_joint(jt, stream, jaux);
            kernels[J[0]] += launch_count() - k0;  // the joint pass is counted on the first instance
            for (cudaStream_t x : jaux) {
                cudaEventRecord(ev, x);
                cudaStreamWaitEvent(stream, ev, 0);
            }
            for (int i : J) kernels[i] += h[i]->sim->joint_post(st, stream);
            for (int i : J) h[i]->sim->join_to(stream);
        }
        for (int i : R) h[i]->sim->join_to(stream);
        launch_count() = count0;  // captured, not launched
        cudaError_t e = cudaStreamEndCapture(stream, &graph);
        if (e != cudaSuccess) { graph = nullptr; return fail(PIC_ERR_CUDA, "batch graph capture: %s", cudaGetErrorString(e)); }
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) { exec = nullptr; return fail(PIC_ERR_CUDA, "batch graph instantiate: %s", cudaGetErrorString(e)); }
        for (size_t i = 0; i < h.size(); i++) epochs[i] = h[i]->sim->graph_epoch();
        return PIC_OK;
    }
    // `to` waits for the work queued on `from` so far
    int order(cudaStream_t from, cudaStream_t to) {
        CUDA_TRY(cudaEventRecord(ev, from));
        CUDA_TRY(cudaStreamWaitEvent(to, ev, 0));
        return PIC_OK;
    }
    int step(long long n) {
        for (auto *x : h) {  // the batch stream starts after everything queued on the instances
            int rc = x->sim->batch_prepare();
            if (rc) return rc;
            rc = order(x->sim->main_stream(), stream);
            if (rc) return rc;
        }
        bool ready = true;
        for (auto *x : h) ready = ready && x->sim->batch_ready();
        while (ready && n >= DFT_BLOCK) {
            if (stale()) {
                int rc = capture();
                if (rc) return rc;
            }
            CUDA_TRY(cudaGraphLaunch(exec, stream));
            for (size_t i = 0; i < h.size(); i++) h[i]->sim->after_block(kernels[i]);
            n -= DFT_BLOCK;
        }
        for (auto *x : h) {  // instance streams wait for the batch; any remainder steps there
            int rc = order(stream, x->sim->main_stream());
            if (rc) return rc;
            if (n > 0) {
                rc = x->sim->step_direct(n);
                if (rc) return rc;
                rc = order(x->sim->main_stream(), stream);
                if (rc) return rc;
            }
        }
        CUDA_TRY(cudaGetLastError());
        return PIC_OK;
    }
    // one whole block of every instance under the current settings, timed on
    // the batch stream (any capture happens before the start event)
    int time_block(cudaEvent_t e0, cudaEvent_t e1, double *us) {
        for (auto *x : h) {
            int rc = x->sim->batch_prepare();
            if (rc) return rc;
            rc = order(x->sim->main_stream(), stream);
            if (rc) return rc;
        }
        if (stale()) {
            int rc = capture();
            if (rc) return rc;
        }
        CUDA_TRY(cudaEventRecord(e0, stream));
        CUDA_TRY(cudaGraphLaunch(exec, stream));
        CUDA_TRY(cudaEventRecord(e1, stream));
        for (size_t i = 0; i < h.size(); i++) h[i]->sim->after_block(kernels[i]);
        for (auto *x : h) {
            int rc = order(stream, x->sim->main_stream());
            if (rc) return rc;
        }
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        *us = 1e3 * ms / DFT_BLOCK;
        return PIC_OK;
    }

    int set_all(const pic_tuning &t) {
        for (auto *x : h) {
            const int rc = x->sim->set_tuning(t);
            if (rc) return rc;
        }
        return PIC_OK;
    }

    // the candidates of pic_tune, each applied to every instance and timed on
    // whole batch blocks
    int tune(int rounds, pic_tune_report *rep) {
        if (rounds < 1 || rounds > 16) return fail(PIC_ERR_ARG, "rounds must be 1..16");
        for (auto *x : h) {  // every instance to its own block boundary
            const int left = x->sim->steps_to_boundary();
            if (left) {
                int rc = x->sim->step_direct(left);
                if (rc) return rc;
            }
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        {
            cudaError_t ce = cudaEventCreate(&e0);
            if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
            if (ce != cudaSuccess) {
                if (e0) cudaEventDestroy(e0);
                return fail(PIC_ERR_CUDA, "tuning events: %s", cudaGetErrorString(ce));
            }
        }
        const int deps[5] = {0, 2048, 4096, 8192, 16384}, everies[4] = {8, 16, 32, 64}, blocks[3] = {128, 256, 512};
        pic_tuning cand[PIC_TUNE_MAX_CANDIDATES];
        double best_us[PIC_TUNE_MAX_CANDIDATES];
        int nc = 0, rc = PIC_OK, win = 0;
        auto pass = [&](int first, int count) -> int {
            for (int r = 0; r < rounds; r++)
                for (int c = first; c < first + count; c++) {
                    int q = set_all(cand[c]);
                    if (q) return q;
                    double us = 0.0;
                    q = time_block(e0, e1, &us);
                    if (q) return q;
                    best_us[c] = std::min(best_us[c], us);
                }
            win = first;
            for (int c = first; c < first + count; c++)
                if (best_us[c] < best_us[win]) win = c;
            return PIC_OK;
        };
        const pic_tuning start = rep_start();
        int cand_lanes[PIC_TUNE_MAX_CANDIDATES];
        const int lanes0 = lanes;
        for (int d : deps) {
            cand_lanes[nc] = lanes0;
            cand[nc] = pic_tuning{d, start.sort_every, start.field_block, start.field_path};
            best_us[nc++] = 1e300;
        }
        rc = pass(0, 5);
        if (!rc) {
            const pic_tuning t = cand[win];
            for (int e : everies) {
                cand_lanes[nc] = lanes0;
                cand[nc] = pic_tuning{t.dep_smem_bytes, e, t.field_block, t.field_path};
                best_us[nc++] = 1e300;
            }
            rc = pass(5, 4);
        }
        if (!rc) {
            const pic_tuning t = cand[win];
            for (int b : blocks) {
                cand_lanes[nc] = lanes0;
                cand[nc] = pic_tuning{t.dep_smem_bytes, t.sort_every, b, t.field_path};
                best_us[nc++] = 1e300;
            }
            rc = pass(9, 3);
        }
        if (!rc && any_fused()) {  // the fused pass (where an instance's grid takes it) against the split updates
            const pic_tuning t = cand[win];
            for (int fp : {1, 0}) {
                cand_lanes[nc] = lanes0;
                cand[nc] = pic_tuning{t.dep_smem_bytes, t.sort_every, t.field_block, fp};
                best_us[nc++] = 1e300;
            }
            rc = pass(12, 2);
        }
        // then how many instances run side by side: 1, 2, 4, 8 chains or all
        int nlanes = 0;
        if (!rc) {
            const pic_tuning t = cand[win];
            const int first = nc;
            for (int l : {1, 2, 4, 8, 0}) {
                if (l >= (int)h.size()) continue;
                cand_lanes[nc] = l;
                cand[nc] = t;
                best_us[nc++] = 1e300;
            }
            nlanes = nc - first;
            for (int r = 0; r < rounds && !rc; r++)
                for (int c = first; c < nc && !rc; c++) {
                    if (lanes != cand_lanes[c]) { lanes = cand_lanes[c]; drop(); }
                    double us = 0.0;
                    rc = time_block(e0, e1, &us);
                    best_us[c] = std::min(best_us[c], us);
                }
            if (!rc) {
                win = first;
                for (int c = first; c < nc; c++)
                    if (best_us[c] < best_us[win]) win = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        rc = set_all(cand[win]);
        if (rc) return rc;
        if (lanes != cand_lanes[win]) { lanes = cand_lanes[win]; drop(); }
        if (rep) {
            std::memset(rep, 0, sizeof(*rep));
            rep->best = cand[win];
            rep->n = nc;
            rep->best_lanes = cand_lanes[win];
            for (int c = 0; c < nc; c++) {
                rep->cand[c] = cand[c];
                rep->us_per_step[c] = best_us[c];
                rep->lanes[c] = cand_lanes[c];
            }
            rep->steps = (long long)rounds * (12 + nlanes) * DFT_BLOCK;
        }
        return PIC_OK;
    }
    // the first instance's sort interval (the box candidates are timed at it)
    pic_tuning rep_start() const {
        pic_tuning t{};
        pic_get_tuning(h[0], &t);
        t.field_path = any_fused() ? 1 : 0;  // the fused pass wherever an instance's grid takes it
        return t;
    }
    bool any_fused() const {
        for (auto *x : h)
            if (x->sim->fused_capable()) return true;
        return false;
    }

    ~pic_batch() {
        if (stream) cudaStreamSynchronize(stream);
        drop();
        if (ev) cudaEventDestroy(ev);
        for (cudaStream_t x : jaux)
            if (x) cudaStreamDestroy(x);
        if (d_tab) cudaFree(d_tab);
        if (d_items) cudaFree(d_items);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

extern "C" {

int pic_batch_create(int n, pic_handle *const *handles, void *stream, pic_batch **out) {
    NvtxRange nvtx_range("pic_batch_create");
    g_err.clear();
    if (!out) return fail(PIC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !handles) return fail(PIC_ERR_ARG, "need at least one handle");
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
    std::unique_ptr<pic_batch> b(new pic_batch());
    for (int i = 0; i < n; i++) {
        if (!handles[i]) return fail(PIC_ERR_ARG, "handle %d is NULL", i);
        for (int q = 0; q < i; q++)
            if (handles[q] == handles[i]) return fail(PIC_ERR_ARG, "handle %d appears twice", i);
        if (handles[i]->sim->device != dev)
            return fail(PIC_ERR_ARG, "handle %d lives on device %d, not on the current device %d", i,
                        handles[i]->sim->device, dev);
        b->h.push_back(handles[i]);
    }
    b->epochs.assign(n, -1);
    b->kernels.assign(n, 0);
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming));
    for (cudaStream_t &x : b->jaux) CUDA_TRY(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    *out = b.release();
    return PIC_OK;
}

int pic_batch_step(pic_batch *b, int64_t nsteps) {
    NvtxRange nvtx_range("pic_batch_step");
    g_err.clear();
    if (!b) return fail(PIC_ERR_ARG, "NULL batch");
    if (nsteps < 0) return fail(PIC_ERR_ARG, "negative step count");
    return b->step(nsteps);
}

int pic_batch_set_lanes(pic_batch *b, int32_t lanes) {
    g_err.clear();
    if (!b) return fail(PIC_ERR_ARG, "NULL batch");
    if (lanes < 0) return fail(PIC_ERR_ARG, "lanes must be >= 0");
    if (lanes != b->lanes) {
        b->lanes = lanes;
        b->drop();
    }
    return PIC_OK;
}

int pic_batch_set_joint(pic_batch *b, int32_t joint) {
    g_err.clear();
    if (!b) return fail(PIC_ERR_ARG, "NULL batch");
    if (joint != 0 && joint != 1) return fail(PIC_ERR_ARG, "joint must be 0 or 1");
    if ((joint != 0) != b->joint) {
        b->joint = joint != 0;
        b->drop();
    }
    return PIC_OK;
}

int pic_batch_tune(pic_batch *b, int32_t rounds, pic_tune_report *report) {
    NvtxRange nvtx_range("pic_batch_tune");
    g_err.clear();
    if (!b) return fail(PIC_ERR_ARG, "NULL batch");
    const int rc = b->tune(rounds, report);
    if (rc) return rc;
    return pic_batch_sync(b);
}

int pic_batch_sync(pic_batch *b) {
    NvtxRange nvtx_range("pic_batch_sync");
    g_err.clear();
    if (!b) return fail(PIC_ERR_ARG, "NULL batch");
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (auto *x : b->h) {
        const int rc = x->precision == PIC_FP64 ? S<double>(x)->sync() : S<float>(x)->sync();
        if (rc) return rc;
    }
    return PIC_OK;
}

int pic_batch_destroy(pic_batch *b) {
    NvtxRange nvtx_range("pic_batch_destroy");
    g_err.clear();
    delete b;
    return PIC_OK;
}

}  // extern "C"
