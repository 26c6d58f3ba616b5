/*
 * FP64 CPU oracle for the scattered-field particle-in-cell (SFF-PIC) step of
 * Lytova et al., "Scattered field formalism in the particle-in-cell method for
 * plasma acceleration in tightly focused ultrashort laser beams" (arXiv 2310.11393).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header, table or
 * helper with the CUDA library; the only thing both sides implement alike is the
 * published SplitMix64 counter generator that places the seeded particles.
 *
 * Units are the paper's dimensionless plasma units (Table "tab:units"): c = 1,
 * omega = k = 1, lengths in lambda/2pi, electron charge -1 and mass 1, densities
 * in n_c.  Everything is double precision.
 *
 * Parity status of each function (what pins it) is stated in the test-suite;
 * nothing here is "parity unpinned".
 */
#ifndef SFFPIC_ORACLE_H
#define SFFPIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BEAM_NONE = 0, ORC_BEAM_PLANE = 1, ORC_BEAM_LP = 2, ORC_BEAM_RP = 3, ORC_BEAM_UNIFORM = 4,
       ORC_BEAM_GAUSS2D = 5 };
/* slab density profile along x: uniform, or the super-Gaussian of Sec. 3.1 */
enum { ORC_PROFILE_UNIFORM = 0, ORC_PROFILE_SUPERGAUSS = 1 };
/* Boris (1970); Vay, Phys. Plasmas 15, 056701 (2008); Higuera & Cary, Phys. Plasmas 24,
 * 052104 (2017) */
enum { ORC_PUSHER_BORIS = 0, ORC_PUSHER_VAY = 1, ORC_PUSHER_HC = 2 };
enum { ORC_ENV_SIN2 = 0, ORC_ENV_GAUSS = 1 };
enum { ORC_BC_MUR = 0, ORC_BC_PERIODIC = 1 };

typedef struct {
    int dim;              /* 1, 2 or 3 resolved axes (x, then y, then z) */
    int n[3];             /* cells per resolved axis */
    double dx;            /* cell size (same on every axis) */
    double dt;            /* time step */
    int field_bc;         /* ORC_BC_MUR (first-order Mur on every face) or ORC_BC_PERIODIC */
    int tf_mode;          /* 0: scattered-field run; 1: total-field run, plane wave injected at x = 0 (dim 1 only) */
    int beam;             /* ORC_BEAM_* */
    int envelope;         /* plane wave envelope: ORC_ENV_SIN2 or ORC_ENV_GAUSS */
    double a0;            /* plane wave field amplitude E0 = B0 */
    double duration;      /* plane wave field-amplitude FWHM */
    double phi0;          /* carrier / constant phase */
    double t_focus;       /* LP/RP: time the pulse peak crosses the focus; Gaussian envelope: centre */
    double focus[3];      /* LP/RP focus (grid coordinates); plane wave: focus[0] is the reference plane */
    double a, s, psi0;    /* LP/RP pulse parameters a, s, Psi_0 (already derived) */
    double e_unif[3], b_unif[3]; /* ORC_BEAM_UNIFORM external fields */
    int slab_lo[3], slab_hi[3];  /* electron slab, cells [lo, hi) per resolved axis */
    double n_e;           /* electron density of the slab */
    int ppc;              /* particles per cell */
    uint64_t seed;        /* SplitMix64 seed */
    int remove_margin;    /* open boxes: a particle whose position is closer than this many cells to a face is removed */
    int pusher;           /* ORC_PUSHER_*: the momentum update of the Lorentz force (Sec. 2 cites all three) */
    double w0;            /* ORC_BEAM_GAUSS2D waist (a0 = E0, duration = FWHM_T, t_focus = t0, focus) */
    int profile;          /* ORC_PROFILE_*: electron weight n_e f(x)/ppc at the particle's initial x */
    int prof_order;       /* super-Gaussian order p */
    double prof_x0;       /* f(x) = 0 for x <= prof_cut, else 2^-[2 (x - prof_x0)/prof_fwhm]^p */
    double prof_fwhm;
    double prof_cut;
    int incident_grid;    /* 1: the incident field is evaluated on the Yee nodes of each component at
                             t^n and gathered with the scattered field (Smilei's prescribed-field
                             route, Sec. 2 last paragraph); 0: at the particle (Sec. 2) */
} orc_config;

typedef struct orc_sim orc_sim;

/* ---- simulation ---------------------------------------------------------------- */
orc_sim* orc_create(const orc_config* cfg);          /* seeded slab particles (may be none), zero scattered field */
void     orc_destroy(orc_sim* s);
void     orc_step(orc_sim* s, int nsteps);
/* the two parts of one step (orc_step runs them in turn): particles (J cleared, gather,
 * incident field, push, move, deposit, exits), then fields (Yee update, step counter) */
void     orc_step_particles(orc_sim* s);
void     orc_step_fields(orc_sim* s);
int64_t  orc_num_particles(const orc_sim* s);          /* alive */
int64_t  orc_num_exits(const orc_sim* s);
int64_t  orc_step_index(const orc_sim* s);
/* replace all particles: x[n][3] (grid coordinates), u[n][3], w[n], id[n] */
void     orc_set_particles(orc_sim* s, int64_t n, const double* x, const double* u, const double* w, const int64_t* id);
void     orc_get_particles(const orc_sim* s, double* x, double* u, double* w, int64_t* id);
/* exited particles: u at exit, weight, id, step of exit */
void     orc_get_exits(const orc_sim* s, double* u, double* w, int64_t* id, int64_t* step);
/* field arrays: 9 components (Ex Ey Ez Bx By Bz Jx Jy Jz), each ext[2]*ext[1]*ext[0]
 * doubles, x fastest, ext[d] = n[d]+1 on a resolved axis and 1 otherwise.
 * Index i along an axis on which the component is staggered means position i+1/2.
 * After a step, J holds that step's J^{n+1/2}. */
void     orc_extents(const orc_sim* s, int ext[3]);
void     orc_get_fields(const orc_sim* s, double* out);
void     orc_set_fields(orc_sim* s, const double* in);
/* energies: [0] scattered EM, [1] total EM (scattered + incident on the grid),
 * [2] kinetic energy of alive electrons, [3] kinetic energy carried out by exits */
void     orc_energies(const orc_sim* s, double out[4]);
/* max |div E - rho_e - rho_ion| over interior nodes (rho_ion = -rho_e at creation) */
double   orc_gauss_residual(const orc_sim* s);
/* electron charge density on the primal nodes (same layout as one field component) */
void     orc_charge_density(const orc_sim* s, double* out);

/* ---- incident fields (grid coordinates, absolute time) -------------------------- */
void orc_incident(const orc_config* cfg, const double x[3], double t, double E[3], double B[3]);
/* beam frame (paper's x, y, z, t relative to focus / focal time), real fields.
 * branch: 0 automatic, 1 closed form only, 2 ring series only */
void orc_lp_field(double a, double s, double psi0, double phi0,
                  double X, double Y, double Z, double tau, int branch, double E[3], double B[3]);
void orc_rp_field(double a, double s, double psi0, double phi0,
                  double X, double Y, double Z, double tau, int branch, double E[3], double B[3]);
/* complex field (real part is the physical field) for the parameter derivation */
void orc_beam_complex(int beam, double a, double s, double psi0, double phi0,
                      double X, double Y, double Z, double tau, int branch,
                      double Ere[3], double Eim[3], double Bre[3], double Bim[3]);

/* ---- pulse parameters ------------------------------------------------------------- */
double orc_a_from_w0(double w0);                          /* k^2 w0^2 = 2(sqrt(1+(ka)^2)-1) */
double orc_focal_fwhm(int beam, double a, double s);      /* field FWHM of the on-axis focal envelope */
double orc_s_from_duration(int beam, double a, double duration);
double orc_psi0_from_a0(int beam, double a, double s, double a0);

/* ---- seeded generator (SplitMix64, Steele/Lea/Flood 2014) ------------------------ */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k);      /* k-th output of the stream seeded with `seed` */

#ifdef __cplusplus
}
#endif
#endif
