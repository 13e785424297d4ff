/*
 * lbm_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow FP64 CPU reference ("the oracle") for the two-phase D2Q9 lattice Boltzmann step
 * with curved-wall schemes of Yu, Li & Wen, "Modified curved boundary scheme for two-phase
 * lattice Boltzmann simulations" (arXiv:1908.09235).  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header or constant table with
 * the CUDA library; the library never links or calls it.
 *
 * Conventions (stated once, used throughout):
 *   node (i, j) sits at position (i, j); linear index n = j*nx + i; periodic in x and y.
 *   D2Q9 directions 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *   Populations are stored as f[alpha*N + n].
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_HBB = 0,        /* halfway bounce-back (Sec. 2.2, Sec. 3.1)                       */
  OR_FH = 1,         /* Filippova-Haenel ghost node, Eqs. (7)-(10)                     */
  OR_MLS = 2,        /* Mei-Luo-Shyy ghost node, Eqs. (7), (8), (10), (11)             */
  OR_BOUZIDI_L = 3,  /* linear interpolated bounce-back, Eq. (12)                      */
  OR_BOUZIDI_Q = 4,  /* quadratic interpolated bounce-back, Eq. (13)                   */
  OR_ZHAO_YONG = 5,  /* single-node scheme, Eq. (14)                                   */
  OR_MOD_A = 6,      /* modified scheme A: MLS + rest-population correction, Eq. (18) */
  OR_MOD_B = 7,      /* modified scheme B: MLS with fictitious density, Eqs. (20)-(22) */
  OR_BAO = 8,        /* Bao et al. fictitious density, Eq. (23)                        */
  OR_BOUZIDI_L_A = 9 /* linear Bouzidi + the Eq. (18) correction                       */
};

enum { OR_EOS_NONE = 0, OR_EOS_EXP = 1, OR_EOS_CS = 2 };

typedef struct {
  double cx, cy, r;
  int32_t solid_outside; /* 0: solid is |x-c| <= r;  1: solid is |x-c| >= r */
  int32_t pad;
} or_circle;

typedef struct {
  int32_t nx, ny;
  int32_t n_circles, pad0;
  const or_circle* circles;
  double wall_q_lo, wall_q_hi; /* >0: row 0 / row ny-1 solid, links into it get this q */
  int32_t eos, scheme;
  double G;                    /* interaction strength in Eq. (16) */
  double psi0, rho0;           /* exponential pseudopotential psi0*exp(-rho0/rho)  */
  double a, b, R, T;           /* Carnahan-Starling EOS, absolute temperature T     */
  double rho_wall;             /* virtual wall density (contact angle)               */
  double gx, gy;               /* body acceleration, force density rho*g             */
  double azim_C, azim_cx, azim_cy; /* force density (C/r) e_theta about (cx, cy)     */
  double tau;
} or_params;

typedef struct or_sim or_sim;

/* ---- building blocks (exposed for pin tests) ---- */
void or_feq(double rho, double ux, double uy, double out[9]);
void or_guo(double tau, double ux, double uy, double Fx, double Fy, double out[9]);
void or_collide_node(const double f[9], double tau, double Fx, double Fy, double out[9]);
double or_psi(const or_params* p, double rho);
double or_cs_pressure(double a, double b, double R, double T, double rho);
void or_force_from_psi(int nx, int ny, double G, const double* psi, double* Fx, double* Fy);
int or_cs_critical(double a, double b, double R, double* Tc, double* rhoc);
int or_cs_coexistence(double a, double b, double R, double T, double* rhoL, double* rhoV);

/* ---- whole simulation ---- */
or_sim* or_create(const or_params* p);
void or_destroy(or_sim* s);
int or_num_links(const or_sim* s);
int or_num_boundary_nodes(const or_sim* s);
void or_flags(const or_sim* s, uint8_t* flags); /* bit0 solid, bit1 boundary node */
void or_links(const or_sim* s, int32_t* node, uint8_t* dir, double* q);
void or_init_fields(or_sim* s, const double* rho, const double* ux, const double* uy);
void or_init_droplet(or_sim* s, double cx, double cy, double R, double W, double rho_in,
                     double rho_out);
void or_step(or_sim* s, int n);
double or_mass(const or_sim* s);
void or_fields(or_sim* s, double* rho, double* ux, double* uy);
void or_get_f(const or_sim* s, double* f);
void or_set_f(or_sim* s, const double* f);
double or_last_leak(const or_sim* s);   /* sum over boundary nodes of Eq. (15) in the last step */
double or_last_max_node_leak(const or_sim* s); /* max |Eq. (15)| after any correction */
long or_fallbacks(const or_sim* s);
/* Threads the per-node loops use: 1 in the serial build, the OpenMP maximum in the -fopenmp
 * build (the same source; test and host-timing infrastructure only). */
int or_num_threads(void);
/* Channel mode for the flow past a cylinder (Sec. 4.2): Zou-He velocity inlet (u_in, 0) at
 * i = 0 and a fully developed outlet at i = nx - 1 (x no longer periodic; y stays periodic).
 * Single-phase flows only (the psi stencil would still wrap in x). */
void or_set_inflow(or_sim* s, double u_in);
/* Momentum-exchange force on all solid nodes during the last step: the sum over cut links of
 * e_a (f*_a(x_b, t) + f_abar(x_b, t+1)), lattice units. */
void or_force(const or_sim* s, double* fx, double* fy);

#ifdef __cplusplus
}
#endif
#endif
