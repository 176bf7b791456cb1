// probe.cu -- prescribed current sources, the end-of-step probe sampling and
// the probe DFT (the spectrum of the field above the film, Sec. IV, Figs. 6-7).
//
// Sampling: after the E update of step n the field E^{n+1} is interpolated at
// every probe (staggered trilinear) and stored as double in a ring of
// DFT_BLOCK slots.  Every DFT_BLOCK steps (and before any read) the ring is
// folded into the FP64 accumulators:
//     F[p][c][f] += dt * sum_s E_c(x_p, t_s) exp(+i 2 pi f t_s),  t_s = (n_s+1) dt.
// The phase of each (slot, frequency) pair is computed once per flush with an
// FP64 sincos of the exact time; for the FP32 state the per-block partial sum
// runs in float (the samples carry FP32 rounding already) and the running
// accumulators stay FP64.
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
        f.jf_flag[((long long)(k / TILE_Z) * g.nt[1] + j / TILE_Y) * g.nt[0] + i / TILE_X] = (int)(step + 1);
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
}

// E component c interpolated at a position given in cell units (double).
template <typename T>
__device__ T probe_value(const Grid<T> &g, const T *F, const double *xi, int c) {
    int i0[3], i1[3];
    T w[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double s = xi[a] - (a == c ? 0.5 : 0.0);
        const double b = floor(s);
        int ib = (int)b;
        w[a] = (T)(s - b);
        int jb = ib + 1;
        const int n = g.n[a];
        if (g.per[a]) {
            ib = ((ib % n) + n) % n;
            jb = ((jb % n) + n) % n;
        } else {
            ib = ib < 0 ? 0 : (ib >= n ? n - 1 : ib);
            jb = jb < 0 ? 0 : (jb >= n ? n - 1 : jb);
        }
        i0[a] = ib;
        i1[a] = jb;
    }
    T v = T(0);
#pragma unroll
    for (int dk = 0; dk < 2; dk++)
#pragma unroll
        for (int dj = 0; dj < 2; dj++)
#pragma unroll
            for (int di = 0; di < 2; di++) {
                const long long e = ((long long)(dk ? i1[2] : i0[2]) * g.n[1] + (dj ? i1[1] : i0[1])) * g.n[0] +
                                    (di ? i1[0] : i0[0]);
                const T wt = (di ? w[0] : T(1) - w[0]) * (dj ? w[1] : T(1) - w[1]) * (dk ? w[2] : T(1) - w[2]);
                v += wt * F[e];
            }
    return v;
}

// Single block: sample the probes for step n, then advance the step counter.
template <typename T>
__global__ void k_step_tail(Grid<T> g, Fields<T> f, Probes<T> pr, long long *step) {
    const long long n = *step;
    const int slot = (int)(n % DFT_BLOCK);
    for (int q = threadIdx.x; q < pr.np * 3; q += blockDim.x) {
        const int p = q / 3, c = q % 3;
        double v = 0.0;
        if (pr.mask & (1u << c)) v = (double)probe_value(g, f.E[c], pr.xyz_cells + 3 * p, c);
        pr.samples[((long long)slot * pr.np + p) * 3 + c] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) *step = n + 1;
}

template <typename T>
void launch_step_tail(const Grid<T> &g, const Fields<T> &f, const Probes<T> &pr, long long *step, cudaStream_t s) {
    int blk = pr.np * 3;
    blk = blk < 32 ? 32 : (blk > 512 ? 512 : ((blk + 31) / 32) * 32);
    k_step_tail<T><<<1, blk, 0, s>>>(g, f, pr, step);
}

// Phase table: phasor[s][f] for the count most recent steps.
__global__ void k_dft_phasor(const double *freq, int nf, double *phasor, const long long *step, int count, double dt) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (f >= nf) return;
    const long long n = *step - count + s;  // the step that produced this sample
    const double t = (double)(n + 1) * dt;
    double sn, cs;
    sincos(2.0 * 3.141592653589793 * freq[f] * t, &sn, &cs);
    phasor[((long long)s * nf + f) * 2] = cs;
    phasor[((long long)s * nf + f) * 2 + 1] = sn;
}

// One thread per (probe, component, frequency): fold the buffered samples.
template <typename A>
__global__ void k_dft_accumulate(const double *samples, const double *phasor, double *F,
                                 int np, int nf, unsigned mask, const long long *step, int count, double dt) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int pc = blockIdx.y;
    const int p = pc / 3, c = pc % 3;
    if (f >= nf || !(mask & (1u << c))) return;
    const long long n0 = *step - count;
    A re = A(0), im = A(0);
    for (int s = 0; s < count; s++) {
        const int slot = (int)((n0 + s) % DFT_BLOCK);
        const A v = (A)samples[((long long)slot * np + p) * 3 + c];
        const A cr = (A)phasor[((long long)s * nf + f) * 2];
        const A ci = (A)phasor[((long long)s * nf + f) * 2 + 1];
        re += v * cr;
        im += v * ci;
    }
    double *out = F + (((long long)p * 3 + c) * nf + f) * 2;
    out[0] += (double)re * dt;
    out[1] += (double)im * dt;
}

template <typename T>
void launch_dft_flush(const Probes<T> &pr, const long long *step, int count, cudaStream_t s) {
    if (count <= 0 || pr.np <= 0 || pr.nf <= 0) return;
    const int blk = 128;
    dim3 g1((pr.nf + blk - 1) / blk, count);
    k_dft_phasor<<<g1, blk, 0, s>>>(pr.freq, pr.nf, pr.phasor, step, count, pr.dt);
    dim3 g2((pr.nf + blk - 1) / blk, pr.np * 3);
    k_dft_accumulate<T><<<g2, blk, 0, s>>>(pr.samples, pr.phasor, pr.F, pr.np, pr.nf, pr.mask, step, count,
                                           pr.dt);
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

}  // namespace pic
