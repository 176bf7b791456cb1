// probe.cu -- prescribed current sources, the end-of-step probe sampling and
// the probe DFT (the spectrum of the field above the film, Sec. IV, Figs. 6-7).
//
// Sampling: after the E update of step n the field E^{n+1} is interpolated at
// every probe (staggered trilinear) and stored as double in a ring of
// DFT_BLOCK slots.  Every DFT_BLOCK steps (and before any read) the ring is
// folded into the FP64 accumulators:
//     F[p][c][f] += dt * sum_s E_c(x_p, t_s) exp(+i 2 pi f t_s),  t_s = (n_s+1) dt.
// The phases of a flush are built in FP64 from the exact time of its first
// step; for the FP32 state the per-block partial sum runs in float (the
// samples carry FP32 rounding already) and the running accumulators stay FP64.
#include "pic_internal.cuh"

namespace pic {

struct SourceList {
    Source s[MAX_SOURCES];
};

template <typename T>
__global__ void k_sources(Grid<T> g, Fields<T> f, SourceList sl, double dt) {
    const Source &s = sl.s[blockIdx.y];
    const long long nb = (long long)(s.box[1] - s.box[0]) * (s.box[3] - s.box[2]) * (s.box[5] - s.box[4]);
    const long long step = *f.step;
    const double t = ((double)step + 0.5) * dt;
    const double x = (t - s.t0) / s.tau;
    const double env = exp(-x * x);
    const double v = s.f0 > 0.0 ? s.amp * env * sin(2.0 * 3.141592653589793 * s.f0 * (t - s.t0))
                                : s.amp * (-2.0 * x) * env;
    const int wi = s.box[1] - s.box[0], wj = s.box[3] - s.box[2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nb; q += (long long)gridDim.x * blockDim.x) {
        const int i = s.box[0] + (int)(q % wi);
        const int j = s.box[2] + (int)((q / wi) % wj);
        const int k = s.box[4] + (int)(q / ((long long)wi * wj));
        const long long e = ((long long)k * g.n[1] + j) * g.n[0] + i;
        atomicAdd(&f.Jf[s.comp][e], (T)v);
        mark_jf_tile(f.jf_flag, f.jf_list, f.jf_count,
                     ((long long)(k / TILE_Z) * g.nt[1] + j / TILE_Y) * g.nt[0] + i / TILE_X, (int)(step + 1));
    }
}

template <typename T>
void launch_sources(const Grid<T> &g, const Fields<T> &f, const Source *src, int nsrc, double dt, cudaStream_t s) {
    if (nsrc <= 0) return;
    SourceList sl;
    long long most = 1;
    for (int q = 0; q < nsrc && q < MAX_SOURCES; q++) {
        sl.s[q] = src[q];
        long long nb = (long long)(src[q].box[1] - src[q].box[0]) * (src[q].box[3] - src[q].box[2]) *
                       (src[q].box[5] - src[q].box[4]);
        if (nb > most) most = nb;
    }
    const int blk = 256;
    long long nblk = (most + blk - 1) / blk;
    if (nblk > 1024) nblk = 1024;
    k_sources<T><<<dim3((unsigned)nblk, (unsigned)nsrc), blk, 0, s>>>(g, f, sl, dt);
    launch_count() += 1;
}

// One block: each warp interpolates whole probes (24 lanes = 3 components x
// 8 corners of the precomputed stencil, summed by shuffles), then thread 0
// advances the step counter once every sample of step n is written.
template <typename T>
__global__ void __launch_bounds__(1024) k_step_tail(Grid<T> g, Fields<T> f, Probes<T> pr, long long *step) {
    pdl_wait();
    pdl_release();
    const long long n = *step;
    const int slot = (int)(n % DFT_BLOCK);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int c = lane >> 3;
    for (int p = warp; p < pr.np; p += nwarps) {
        T v = T(0);
        if (c < 3 && (pr.mask & (1u << c))) {
            const long long q = (long long)p * 24 + lane;
            v = pr.st_w[q] * f.E[c][pr.st_idx[q]];
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off, 8);
        if ((lane & 7) == 0 && c < 3) pr.samples[((long long)slot * pr.np + p) * 3 + c] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *step = n + 1;
        *f.jf_count = 0;  // the J_f tile list of the next step starts empty
    }
}

template <typename T>
void launch_step_tail(const Grid<T> &g, const Fields<T> &f, const Probes<T> &pr, long long *step, cudaStream_t s) {
    int blk = 32 * pr.np;
    blk = blk < 32 ? 32 : (blk > 1024 ? 1024 : blk);
    launch_pdl(k_step_tail<T>, dim3(1), dim3(blk), 0, s, g, f, pr, step);
    launch_count() += 1;
}

// Phase table phasor[s][f] = exp(+i 2 pi f (n_s+1) dt) for the count most
// recent steps.  A thread covers PHASE_RUN consecutive steps of one
// frequency: one FP64 sincos for its first step and one for the per-step
// rotation, then a complex product per step (error below 1e-15 per run).
constexpr int PHASE_RUN = 8;

__global__ void k_dft_phasor(const double *freq, int nf, double *phasor, const long long *step, int count, double dt) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int s0 = blockIdx.y * PHASE_RUN;
    if (f >= nf || s0 >= count) return;
    const long long n0 = *step - count;  // the step that produced slot s = 0
    const double w = 2.0 * 3.141592653589793 * freq[f];
    double zr, zi, rr, ri;
    sincos(w * ((double)(n0 + s0 + 1) * dt), &zi, &zr);
    sincos(w * dt, &ri, &rr);
    const int s1 = s0 + PHASE_RUN < count ? s0 + PHASE_RUN : count;
    for (int s = s0; s < s1; s++) {
        phasor[((long long)s * nf + f) * 2] = zr;
        phasor[((long long)s * nf + f) * 2 + 1] = zi;
        const double tr = zr * rr - zi * ri;
        zi = zr * ri + zi * rr;
        zr = tr;
    }
}

// Fold the buffered samples into the FP64 accumulators.  A thread owns one
// frequency and DFT_ROWS (probe, component) rows of a block; the block's
// samples sit in shared memory, so each phase is read once per thread.
constexpr int DFT_ROWS = 16;

template <typename A>
__global__ void __launch_bounds__(128) k_dft_accumulate(const double *samples, const double *phasor, double *F, int np,
                                                        int nf, unsigned mask, const long long *step, int count,
                                                        double dt) {
    __shared__ A s_smp[DFT_BLOCK][DFT_ROWS];
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int row0 = blockIdx.y * DFT_ROWS;
    const int nrows = np * 3;
    const long long n0 = *step - count;
    for (int q = threadIdx.x; q < count * DFT_ROWS; q += blockDim.x) {
        const int s = q / DFT_ROWS, r = q % DFT_ROWS;
        const int slot = (int)((n0 + s) % DFT_BLOCK);
        s_smp[s][r] = (row0 + r < nrows) ? (A)samples[(long long)slot * nrows + row0 + r] : A(0);
    }
    __syncthreads();
    if (f >= nf) return;
    A re[DFT_ROWS], im[DFT_ROWS];
#pragma unroll
    for (int r = 0; r < DFT_ROWS; r++) re[r] = im[r] = A(0);
    for (int s = 0; s < count; s++) {
        const A cr = (A)phasor[((long long)s * nf + f) * 2];
        const A ci = (A)phasor[((long long)s * nf + f) * 2 + 1];
#pragma unroll
        for (int r = 0; r < DFT_ROWS; r++) {
            re[r] += s_smp[s][r] * cr;
            im[r] += s_smp[s][r] * ci;
        }
    }
#pragma unroll
    for (int r = 0; r < DFT_ROWS; r++) {
        const int row = row0 + r;
        if (row >= nrows || !(mask & (1u << (row % 3)))) continue;
        double *out = F + ((long long)row * nf + f) * 2;
        out[0] += (double)re[r] * dt;
        out[1] += (double)im[r] * dt;
    }
}

template <typename T>
void launch_dft_flush(const Probes<T> &pr, const long long *step, int count, cudaStream_t s) {
    if (count <= 0 || pr.np <= 0 || pr.nf <= 0) return;
    const int blk = 128;
    k_dft_phasor<<<dim3((pr.nf + blk - 1) / blk, (count + PHASE_RUN - 1) / PHASE_RUN), blk, 0, s>>>(
        pr.freq, pr.nf, pr.phasor, step, count, pr.dt);
    launch_count() += 1;
    dim3 g2((pr.nf + blk - 1) / blk, (pr.np * 3 + DFT_ROWS - 1) / DFT_ROWS);
    k_dft_accumulate<T><<<g2, blk, 0, s>>>(pr.samples, pr.phasor, pr.F, pr.np, pr.nf, pr.mask, step, count, pr.dt);
    launch_count() += 1;
}

template void launch_sources<float>(const Grid<float> &, const Fields<float> &, const Source *, int, double,
                                    cudaStream_t);
template void launch_sources<double>(const Grid<double> &, const Fields<double> &, const Source *, int, double,
                                     cudaStream_t);
template void launch_step_tail<float>(const Grid<float> &, const Fields<float> &, const Probes<float> &, long long *,
                                      cudaStream_t);
template void launch_step_tail<double>(const Grid<double> &, const Fields<double> &, const Probes<double> &,
                                       long long *, cudaStream_t);
template void launch_dft_flush<float>(const Probes<float> &, const long long *, int, cudaStream_t);
template void launch_dft_flush<double>(const Probes<double> &, const long long *, int, cudaStream_t);

// Space-time spectrum of the probe line (the dispersion picture of Sec. II,
// Fig. 2): out[q][f] = |sum_p F[p][comp][f] exp(-i k_q s_p)|^2, s_p the
// probe coordinate along the line's axis.  One thread per (k, f); FP64.
__global__ void k_probe_kw(const double *F, const double *xyz_cells, double cell, int axis, int np, int nf,
                           int comp, const double *k, int nk, double *out) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (f >= nf || q >= nk) return;
    double re = 0.0, im = 0.0;
    for (int p = 0; p < np; p++) {
        const double sp = xyz_cells[3 * p + axis] * cell;
        double sn, cs;
        sincos(-k[q] * sp, &sn, &cs);
        const double *z = F + (((long long)p * 3 + comp) * nf + f) * 2;
        re += z[0] * cs - z[1] * sn;
        im += z[0] * sn + z[1] * cs;
    }
    out[(long long)q * nf + f] = re * re + im * im;
}

void launch_probe_kw(const double *F, const double *xyz_cells, double cell, int axis, int np, int nf, int comp,
                     const double *k, int nk, double *out, cudaStream_t s) {
    const int blk = 128;
    k_probe_kw<<<dim3((nf + blk - 1) / blk, nk), blk, 0, s>>>(F, xyz_cells, cell, axis, np, nf, comp, k, nk, out);
    launch_count() += 1;
}

}  // namespace pic
