/*
 * PBD-R reference oracle: plain, slow, serial FP64 CPU implementation of one
 * PBD-R substep (Algorithm 1 of "Physically Accurate Rigid-Body Dynamics in
 * Particle-Based Simulation", arXiv 2603.14634) and of the neighbour search it
 * relies on.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA implementation.
 *
 * Units: SI.  State is FP64 except where the method fixes FP32: the neighbour
 * predicate and cell keys are evaluated on FP32 positions with FP32
 * round-to-nearest arithmetic and no contraction (the file is compiled with
 * -ffp-contract=off), so that both implementations make the same decisions.
 */
#ifndef PBDR_ORACLE_H
#define PBDR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* flags (same bit meanings as the library's scene flags) */
#define ORC_STD_VELOCITY (1u << 0) /* V = (X - X_init)/dt instead of the incremental update */
#define ORC_NO_LINMOM    (1u << 1) /* skip the linear-momentum correction  */
#define ORC_NO_ANGMOM    (1u << 2) /* skip the angular-momentum correction */
#define ORC_CONTACT_AVG  (1u << 3) /* average particle-particle corrections */
#define ORC_SM_FROM_XI   (1u << 4) /* shape matching on X_i, not X_i + contact corrections */

typedef struct {
  int32_t num_particles;
  int32_t num_bodies;
  const int32_t *body_off; /* [B+1] body b owns particles [body_off[b], body_off[b+1]) */
  const double *inv_mass;  /* [N] w_p > 0 */
  const double *rest;      /* [N*3] rest offsets q_p = x0_p - c0 (orc_rest_shape) */
  const double *body_mass; /* [B] M_b */
  double radius;           /* r */
  double friction;         /* mu (kinetic = static) */
  double gravity[3];
  double plane[4];         /* n (unit), d : ground is n.x = d, solid side n.x < d */
  double dt;
  int32_t iterations;      /* solver iterations K */
  uint32_t flags;
  const double *force;     /* [B*3] constant force at the CoM, or NULL */
  const double *torque;    /* [B*3] constant torque about the CoM, or NULL */
} orc_scene;

/* FP32 constants of the neighbour search derived from the particle radius:
 * Rn = (float)(2.2*(double)r), Rn2 = Rn*Rn (FP32), h = (float)(Rn*(1+2^-10)),
 * inv_h = (float)(1/(double)h). */
void orc_nbr_constants(float radius, float *Rn, float *Rn2, float *h, float *inv_h);

/* hash-table size of a scene of n particles: smallest power of two >= 2n */
uint32_t orc_table_size(int32_t n);

/* bucket of every particle: Teschner et al. 2003 prime-XOR hash of the FP32
 * cell coordinates, masked to the table size T (a power of two) */
void orc_cell_keys(int32_t n, const float *x, float inv_h, uint32_t T, uint32_t *key);

/* stable sort of (key, particle id) pairs by key; ids ascending within a key */
void orc_sort_keys(int32_t n, const uint32_t *key, uint32_t T,
                   uint32_t *sorted_key, uint32_t *sorted_id);

/* neighbour lists: N(p) = { q != p : body(q) != body(p), d2_fp32(x_p, x_q) < Rn2 }
 * as ascending CSR (off[n+1], idx).  Returns the total count; entries beyond
 * `cap` are counted but not written. */
int64_t orc_neighbors_brute(int32_t n, const float *x, const int32_t *body,
                            float Rn2, int32_t *off, int32_t *idx, int64_t cap);
int64_t orc_neighbors_grid(int32_t n, const float *x, const int32_t *body,
                           float Rn2, float inv_h, int32_t *off, int32_t *idx,
                           int64_t cap);

/* rest shape: M_b = sum m_p, c0_b = sum m_p x_p / M_b, q_p = x_p - c0_b */
void orc_rest_shape(int32_t n, int32_t nb, const int32_t *body_off,
                    const double *inv_mass, const double *x0, double *rest,
                    double *body_mass);

/* rotation part R of A (row-major 3x3): the proper rotation maximising
 * tr(R^T A), via an SVD from a Jacobi eigen-decomposition of A^T A.  Rank <= 1
 * inputs return Rprev. */
void orc_polar_rotation(const double *A, const double *Rprev, double *R);

/* inertia tensor about the centre of mass c of n particles:
 * I = sum m (|r|^2 I3 - r r^T), r = x - c (row-major 3x3) */
void orc_body_inertia(int32_t n, const double *x, const double *mass,
                      const double *c, double *I);

/* momentum enforcement for one body (Eqs. lin_momentum and ang_momentum):
 * given the states before (xb, vb) and after (xa, va) shape matching, writes
 * the corrected x, v (may alias xa, va). */
void orc_enforce_momentum(int32_t n, const double *mass, const double *xb,
                          const double *vb, const double *xa, const double *va,
                          double dt, uint32_t flags, double *x_out, double *v_out);

/* one PBD-R substep of one scene, in place on x, v ([N*3]).  rot ([B*9],
 * row-major) holds each body's last shape-matching rotation (warm start for
 * degenerate bodies; identity at creation) and is updated.  use_brute selects
 * the O(N^2) neighbour search.  Returns 0, or -1 on allocation failure. */
int orc_substep(const orc_scene *s, double *x, double *v, double *rot, int use_brute);

#ifdef __cplusplus
}
#endif

#endif
