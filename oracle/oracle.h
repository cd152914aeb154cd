/* Plain FP64 CPU oracle of the cut-cell step (test infrastructure only).
 * Used by tests/, the smoke check and the benchmark's CPU-baseline leg. */
#ifndef CUTCELL_ORACLE_H
#define CUTCELL_ORACLE_H
#include <stdint.h>

enum { OC_OK = 0, OC_EINVAL = 1, OC_EGEOM = 3 };
enum { OC_F_RHOP = 0, OC_F_PP = 1, OC_F_MX = 2, OC_F_MY = 3, OC_F_MZ = 4, OC_F_UB = 5 };
/* derived output fields */
enum { OC_D_U = 0, OC_D_V = 1, OC_D_W = 2, OC_D_THETA = 3 };

typedef struct {
  int nx, ny, nz;
  double dx, dy, dz;
  double dt;
  double U, N, theta0, p_surf, p0, g, R, cp;
  double ra_nu, c4, sponge_frac, tau_max;
  int bc_slip;
  double ztop;  /* height of the domain top for the sponge; 0: nz*dz */
} oc_params;

/* refined level l >= 1: nx, ny, nz cells of spacing 2^-l H starting at the
 * floor; its cell i covers the cell (i + ox)/2 of level l-1 */
typedef struct { int nx, ny, nz, ox, oy; } oc_box;

typedef struct oc_model oc_model;

oc_model *oc_create(const oc_params *P, const double *h, int *status);
void oc_destroy(oc_model *m);
void oc_init_state(oc_model *m);
void oc_step(oc_model *m, int nsteps);
int oc_dims(const oc_model *m, long *ncell, long *ncorner, long *ncol, int *gz);
int oc_get_state(oc_model *m, int field, int level, double *out);
int oc_set_state(oc_model *m, int field, int level, const double *in);
int oc_get_state_padded(oc_model *m, int field, int level, double *out);
void oc_padding(const oc_model *m, int *g, int *nxp, int *nyp, int *nzp);
int oc_get_geometry(const oc_model *m, double *vf, double *ax, double *ay, double *az, int8_t *cls,
                    int32_t *root, double *vg, double *hc, double *gx, double *gy);
int oc_get_points(const oc_model *m, int8_t *vcls, int32_t *bK, int32_t *bI, int32_t *bJ, double *ba,
                  double *bb, double *bn, int32_t *mK, double *mg);
int oc_base_len(const oc_model *m);
int oc_get_base(const oc_model *m, double *rhob, double *pb, int *koff, int *nb);
double oc_mass(const oc_model *m, int level);
int oc_nsteps(const oc_model *m);
double oc_heat(const oc_model *m, int level);
int oc_get_derived(const oc_model *m, int which, int level, double *out);
int oc_error_norms(const oc_model *a, const oc_model *b, int which, double zmin, double *out);

double oc_line_int(double z, double ha, double hb, double len);
double oc_line_frac(double z, double ha, double hb);
double oc_col_int(double z, double h00, double h10, double h01, double h11, double dx, double dy,
                  int kind);
double oc_gauss_legendre8(double (*f)(double, void *), void *ctx, double a, double b);

typedef struct oc_refine oc_refine;
oc_refine *oc_refine_create(const oc_params *P0, int nlev, const oc_box *boxes, const double *h_finest,
                            int *status);
void oc_refine_destroy(oc_refine *R);
void oc_refine_init(oc_refine *R);
void oc_refine_step(oc_refine *R, int n);
oc_model *oc_refine_level(oc_refine *R, int l);
double oc_refine_mass(oc_refine *R, int both);

#endif
