/* pic_adjoint.h -- gradient of a film's plasmon signal with respect to its
 * Drude parameters, by a hand-written adjoint of the field step.
 *
 * The paper has no adjoint; this serves design studies built on its film
 * model (Sec. III): how the spectral energy of the surface plasmon seen by a
 * probe changes with a per-cell relaxation of the film (a mask m in [0,1]
 * scaling wp^2 in each cell of a design slab), with wp and with gamma.
 *
 * Forward model (one step n -> n+1: the field part of the PIC step of
 * pic.h, with the electrons replaced by a rigid prescribed bunch):
 *   H^{n+1/2} = H^{n-1/2} - dt/mu0 curl E^n                    (CPML on all faces)
 *   J^{n+1}   = kJ J^n + bJ E^n        on every edge touching the design slab  (Eq. 6)
 *   E^{n+1}   = E^n + dt/eps0 [curl H^{n+1/2} - J^{n+1} - Js^{n+1/2}]          (Eq. 8)
 * with kJ = (2 - gamma dt)/(2 + gamma dt), bJ = 2 dt eps0 wp_e^2/(2 + gamma dt),
 * wp_e^2 = wp^2 x (mean of m over the four cells around the edge; m = 0 outside
 * the slab), eps_inf = 1, tangential E held at 0 on the low faces, and Js the
 * current of a rigid Gaussian bunch (charge q, rms radius sigma) moving along
 * +x at speed v:
 *   Js_x(x, t) = q v (2 pi sigma^2)^{-3/2} exp(-|x - x0 - v t e_x|^2 / (2 sigma^2)),
 * evaluated on every Ex edge of the grid at t = (n + 1/2) dt (no truncation:
 * the current is zero only where the Gaussian underflows in FP64).
 * Loss:  L = |F|^2,  F = sum_n E_c(x_p, t_{n+1}) exp(+i omega0 t_{n+1}) dt,
 * E_c interpolated trilinearly on its staggered lattice at the probe x_p
 * (the probe DFT of pic_probe_dft at one frequency).
 *
 * Backward: the transposed step runs from n = N-1 down to 0 on adjoint
 * fields; every E^n and J^n on the design edges is kept in device memory
 * during the forward run (nsteps x design edges x 2 values), so nothing is
 * recomputed.  Gradients are accumulated and reduced in FP64.  Every function
 * returns 0 (PIC_OK) or a negative PIC_ERR_* code of pic.h, with text in
 * pic_last_error(). */
#ifndef PIC_ADJOINT_H
#define PIC_ADJOINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int64_t nx, ny, nz;     /* cells; x fastest in every array */
    double dx;              /* cubic cells [m] */
    double dt;              /* [s]; must satisfy the CFL bound with the Drude term */
    int32_t precision;      /* PIC_FP32 or PIC_FP64 (field state; gradients are FP64) */
    int32_t cpml_cells;     /* CPML on all six faces */
    double cpml_order, cpml_sigma_fac, cpml_kappa_max, cpml_alpha_max;
    double eps0, mu0;
    int64_t design_k0, design_k1;        /* design slab: cell planes [k0, k1), all x and y */
    double bunch_q, bunch_sigma, bunch_v;  /* [C], [m], [m/s] */
    double bunch_x0, bunch_y0, bunch_z0;   /* centre at t = 0 [m] */
    double probe[3];        /* [m] */
    int32_t probe_comp;     /* 0..2: Ex, Ey, Ez */
    int32_t flags;          /* bit 0: keep the one-cell-per-thread kernels where the FP32
                               four-cell ones would run (nx and cpml_cells multiples of 4);
                               bit 1: checkpoint mode (below) */
    double omega0;          /* loss frequency [rad/s] */
    int64_t nsteps;         /* steps of a forward run; nsteps x nx <= 2^28 (the bunch's
                               per-step factors are tabulated at create) */
} pic_adj_config;

typedef struct pic_adj pic_adj;

/* Validate the configuration, build the CPML profiles, the design-edge lists
 * and the probe stencil, and allocate the field state, the adjoint state and
 * the per-step storage on the current device.  Errors: PIC_ERR_ARG,
 * PIC_ERR_CFL (checked with the largest wp a later forward may use is not
 * known here, so only the vacuum bound), PIC_ERR_OOM, PIC_ERR_CUDA. */
int pic_adj_create(const pic_adj_config *cfg, pic_adj **out);

/* Number of mask cells: nx * ny * (design_k1 - design_k0), ordered [k][j][i]. */
int pic_adj_mask_size(const pic_adj *a, int64_t *n);

/* Run the forward model from zero fields for nsteps with the given mask
 * (host array of pic_adj_mask_size values in [0, 1]), wp [rad/s] and gamma
 * [1/s]; returns L and keeps what pic_adj_backward needs.  Errors:
 * PIC_ERR_ARG (NULL, mask outside [0,1], wp or gamma negative), PIC_ERR_CFL
 * (the Drude term breaks the time-step bound), PIC_ERR_CUDA.  Synchronises. */
int pic_adj_forward(pic_adj *a, const double *mask, double wp, double gamma, double *loss);

/* Gradients of the L of the last forward run: dmask (host, mask size), dwp,
 * dgamma.  Errors: PIC_ERR_STATE without a forward run.  Synchronises.
 *
 * Checkpoint mode (flags bit 1): instead of every step's E^n and J^n on the
 * design edges, the forward run keeps the whole field state (E, H, J, CPML
 * memory) every C = 64 ceil(sqrt(nsteps) / 64) steps, and the backward run
 * recomputes each segment of C steps from its checkpoint before running it
 * backward.  Memory: (ceil(nsteps / C) - 1) field states + C steps of design
 * edges instead of nsteps steps of design edges; time: one more forward run.
 * The results are those of the default mode (the same forward arithmetic). */
int pic_adj_backward(pic_adj *a, double *dmask, double *dwp, double *dgamma);

/* Release everything.  NULL is accepted. */
int pic_adj_destroy(pic_adj *a);

#ifdef __cplusplus
}
#endif

#endif /* PIC_ADJOINT_H */
