/*
 * ct.c -- constrained transport of the magnetic field on 2D/3D grids
 * (Sec. 4: "Magnetic field divergence free constraint is preserved by using the
 * CT method, where electromotive forces were averaged according to the
 * CT-contact formalism" of Gardiner & Stone 2005).  TEST INFRASTRUCTURE ONLY
 * (the oracle; see oracle.h).
 *
 * Staggered field: b_d, the component of B normal to the faces of direction d
 * (d < ndim), one value per face, stored like the fluxes of direction d
 * ([m2][m1][m0] with m = n + e_d), the directions one after the other.  In 2D, B_z
 * stays cell-centred and is updated by its fluxes.
 *
 * Edge EMF E_e (e = a x b cyclic) at the edge between cells (ia-1, ia) along a and
 * (ib-1, ib) along b:
 *   E_e = 1/4 [E(a-face, ib-1) + E(a-face, ib) + E(b-face, ia-1) + E(b-face, ia)]
 *       + 1/4 (Lb - Ub) + 1/4 (La - Ra)                           (G&S 2005 Eq. 41)
 * with E = -F^a(B_b) at a-faces, +F^b(B_a) at b-faces, the cell-centre reference
 * E_ref = v_b B_a - v_a B_b, and the contact-upwinded half-cell differences
 *   Lb = up(F^a_D at a-face row ib-1; E(b-face,c) - E_ref(c, ib-1)),
 *   Ub = up(F^a_D at a-face row ib;   E_ref(c, ib) - E(b-face,c)),
 *   La = up(F^b_D at b-face column ia-1; E(a-face,r) - E_ref(ia-1, r)),
 *   Ra = up(F^b_D at b-face column ia;   E_ref(ia, r) - E(a-face,r)),
 * where up(f; x) takes x of the cell on the upwind side of the mass flux f (the
 * lower index if f > 0, the upper if f < 0, their mean if f = 0) (G&S Eq. 50).
 * Face update, d-faces: b_d -= dt (curl E)_d = dt (dE_b/de - dE_e/db)... written
 * out per direction below; the RK3 stages combine b as they combine U.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static int map_i(int c, int n, int bc)
{
    if (bc == OR_BC_PERIODIC) {
        int m = c % n;
        return m < 0 ? m + n : m;
    }
    return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

static int64_t cell_of(const or_grid* g, const int p[3])
{
    int q[3];
    for (int d = 0; d < 3; d++) q[d] = map_i(p[d], g->n[d], g->bc[d]);
    return ((int64_t)q[2] * g->n[1] + q[1]) * g->n[0] + q[0];
}

/* Offset of the faces of direction d in a face-field array, and one face's index. */
int64_t or_ct_face_base(const or_grid* g, int d)
{
    int64_t base = 0;
    for (int e = 0; e < d; e++) {
        int m[3] = {g->n[0], g->n[1], g->n[2]};
        m[e] += 1;
        base += (int64_t)m[0] * m[1] * m[2];
    }
    return base;
}

int64_t or_ct_nfaces(const or_grid* g) { return or_ct_face_base(g, g->ndim); }

static int64_t face_at(const or_grid* g, int d, const int p[3])
{
    /* p[d] in [0, n_d] is the face index along d; the other indices are cells
     * (mapped through the boundaries) */
    int m[3] = {g->n[0], g->n[1], g->n[2]};
    m[d] += 1;
    int q[3];
    for (int e = 0; e < 3; e++) q[e] = (e == d) ? p[e] : map_i(p[e], g->n[e], g->bc[e]);
    return ((int64_t)q[2] * m[1] + q[1]) * m[0] + q[0];
}

/* Face field from cell-centred B: the mean of the two cells next to each face
 * (an initial guess; divergence-free data should come from a vector potential). */
void or_ct_faces_from_cells(const or_grid* g, const double* V, double* bface)
{
    int64_t N = (int64_t)g->n[0] * g->n[1] * g->n[2];
    for (int d = 0; d < g->ndim; d++) {
        int64_t base = or_ct_face_base(g, d);
        int m[3] = {g->n[0], g->n[1], g->n[2]};
        m[d] += 1;
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    int pl[3] = {i, j, k}, pr[3] = {i, j, k};
                    pl[d] -= 1;
                    double bl = V[(5 + d) * N + cell_of(g, pl)];
                    double br = V[(5 + d) * N + cell_of(g, pr)];
                    bface[base + ((int64_t)k * m[1] + j) * m[0] + i] = 0.5 * (bl + br);
                }
    }
}

/* Cell-centred B_d = mean of the two faces of direction d (d < ndim). */
void or_ct_cells_from_faces(const or_grid* g, const double* bface, double* U, double* V)
{
    int64_t N = (int64_t)g->n[0] * g->n[1] * g->n[2];
    for (int d = 0; d < g->ndim; d++) {
        int64_t base = or_ct_face_base(g, d);
        for (int k = 0; k < g->n[2]; k++)
            for (int j = 0; j < g->n[1]; j++)
                for (int i = 0; i < g->n[0]; i++) {
                    int pl[3] = {i, j, k}, pr[3] = {i, j, k};
                    pr[d] += 1;
                    double b = 0.5 * (bface[base + face_at(g, d, pl)] + bface[base + face_at(g, d, pr)]);
                    int64_t c = ((int64_t)k * g->n[1] + j) * g->n[0] + i;
                    if (U) U[(5 + d) * N + c] = b;
                    if (V) V[(5 + d) * N + c] = b;
                }
    }
}

/* In a periodic direction d the faces at index 0 and n_d are the same face: copy
 * face 0 onto face n_d so that both copies hold the same bits (the PVM products
 * would amplify any difference by 1/eps). */
void or_ct_canonical(const or_grid* g, double* bface)
{
    for (int d = 0; d < g->ndim; d++) {
        if (g->bc[d] != OR_BC_PERIODIC) continue;
        int64_t base = or_ct_face_base(g, d);
        int m[3] = {g->n[0], g->n[1], g->n[2]};
        m[d] += 1;
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    int p[3] = {i, j, k};
                    if (p[d] != g->n[d]) continue;
                    int q[3] = {i, j, k};
                    q[d] = 0;
                    bface[base + ((int64_t)k * m[1] + j) * m[0] + i] =
                        bface[base + ((int64_t)q[2] * m[1] + q[1]) * m[0] + q[0]];
                }
    }
}

/* Discrete divergence sum_d (b_d(right) - b_d(left))/dx_d of every cell. */
void or_ct_div(const or_grid* g, const double* bface, double* div)
{
    for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
            for (int i = 0; i < g->n[0]; i++) {
                double s = 0.0;
                for (int d = 0; d < g->ndim; d++) {
                    int64_t base = or_ct_face_base(g, d);
                    int pl[3] = {i, j, k}, pr[3] = {i, j, k};
                    pr[d] += 1;
                    s = s + (bface[base + face_at(g, d, pr)] - bface[base + face_at(g, d, pl)]) / g->dx[d];
                }
                div[((int64_t)k * g->n[1] + j) * g->n[0] + i] = s;
            }
}

static double upwind(double f, double xlo, double xhi)
{
    if (f > 0.0) return xlo;
    if (f < 0.0) return xhi;
    return 0.5 * (xlo + xhi);
}

/* E_e at the edge (ia, ib) (between cells ia-1, ia along a and ib-1, ib along b),
 * pos[e] the cell index along the edge.  Fh[d]: face fluxes of direction d
 * ([12][faces]); V: cell primitives. */
static double edge_emf(const or_grid* g, int e, const int pos[3], double* const Fh[3],
                       const double* V)
{
    const int a = (e + 1) % 3, b = (e + 2) % 3;
    int64_t N = (int64_t)g->n[0] * g->n[1] * g->n[2];
    int ma[3] = {g->n[0], g->n[1], g->n[2]}, mb[3] = {g->n[0], g->n[1], g->n[2]};
    ma[a] += 1;
    mb[b] += 1;
    int64_t NFa = (int64_t)ma[0] * ma[1] * ma[2], NFb = (int64_t)mb[0] * mb[1] * mb[2];
    /* a-faces at index ia along a, rows ib-1 and ib along b */
    int pa0[3] = {pos[0], pos[1], pos[2]}, pa1[3] = {pos[0], pos[1], pos[2]};
    pa0[b] -= 1;
    int64_t fa0 = face_at(g, a, pa0), fa1 = face_at(g, a, pa1);
    /* b-faces at index ib along b, columns ia-1 and ia along a */
    int pb0[3] = {pos[0], pos[1], pos[2]}, pb1[3] = {pos[0], pos[1], pos[2]};
    pb0[a] -= 1;
    int64_t fb0 = face_at(g, b, pb0), fb1 = face_at(g, b, pb1);
    double Ea0 = -Fh[a][(5 + b) * NFa + fa0], Ea1 = -Fh[a][(5 + b) * NFa + fa1];
    double Eb0 = Fh[b][(5 + a) * NFb + fb0], Eb1 = Fh[b][(5 + a) * NFb + fb1];
    double ma0 = Fh[a][fa0], ma1 = Fh[a][fa1];   /* mass fluxes (component D) */
    double mb0 = Fh[b][fb0], mb1 = Fh[b][fb1];
    /* cell-centre reference EMFs of the four cells around the edge:
     * c00 = (ia-1, ib-1), c10 = (ia, ib-1), c01 = (ia-1, ib), c11 = (ia, ib) */
    double Er[2][2];
    for (int s = 0; s < 2; s++)
        for (int r = 0; r < 2; r++) {
            int p[3] = {pos[0], pos[1], pos[2]};
            p[a] += s - 1;
            p[b] += r - 1;
            int64_t c = cell_of(g, p);
            double va = V[(1 + a) * N + c], vb = V[(1 + b) * N + c];
            double Ba = V[(5 + a) * N + c], Bb = V[(5 + b) * N + c];
            Er[s][r] = vb * Ba - va * Bb;
        }
    double Lb = upwind(ma0, Eb0 - Er[0][0], Eb1 - Er[1][0]);
    double Ub = upwind(ma1, Er[0][1] - Eb0, Er[1][1] - Eb1);
    double La = upwind(mb0, Ea0 - Er[0][0], Ea1 - Er[0][1]);
    double Ra = upwind(mb1, Er[1][0] - Ea0, Er[1][1] - Ea1);
    return 0.25 * (((Ea0 + Ea1) + Eb0) + Eb1) + 0.25 * (Lb - Ub) + 0.25 * (La - Ra);
}

/* Number of edges of direction e: n + 1 in the two other directions (2D: e = z only). */
static void edge_dims(const or_grid* g, int e, int m[3])
{
    for (int d = 0; d < 3; d++) m[d] = g->n[d] + ((d != e && d < g->ndim) ? 1 : 0);
}

/* One stage of the face field (Sec. 3.1 stages applied to b):
 *   bout = a b0 + bw (bs - dt (curl E)),  stage weights as for U.
 * Fh: this stage's face fluxes; V: the stage's input primitives. */
void or_ct_stage(const or_grid* g, int stage, double dt, double* const Fh[3], const double* V,
                 const double* b0, const double* bs, double* bout)
{
    double ca = 0.0, cb = 1.0;
    if (stage == 2) { ca = 0.75; cb = 0.25; }
    if (stage == 3) { ca = 1.0 / 3.0; cb = 2.0 / 3.0; }
    /* edge EMFs: 2D only E_z; 3D all three */
    double* E[3] = {0, 0, 0};
    int em[3][3];
    for (int e = 0; e < 3; e++) {
        if (g->ndim == 2 && e != 2) continue;
        edge_dims(g, e, em[e]);
        E[e] = (double*)malloc(sizeof(double) * (size_t)em[e][0] * em[e][1] * em[e][2]);
        for (int k = 0; k < em[e][2]; k++)
            for (int j = 0; j < em[e][1]; j++)
                for (int i = 0; i < em[e][0]; i++) {
                    int pos[3] = {i, j, k};
                    E[e][((int64_t)k * em[e][1] + j) * em[e][0] + i] = edge_emf(g, e, pos, Fh, V);
                }
    }
    /* faces: (curl E)_d = dE_{d+2}/d x_{d+1} - dE_{d+1}/d x_{d+2} (cyclic) */
    for (int d = 0; d < g->ndim; d++) {
        int64_t base = or_ct_face_base(g, d);
        int m[3] = {g->n[0], g->n[1], g->n[2]};
        m[d] += 1;
        const int p1 = (d + 1) % 3, p2 = (d + 2) % 3;
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    int pos[3] = {i, j, k};
                    double curl = 0.0;
                    if (E[p2]) {   /* + dE_{p2}/dx_{p1}: edges of direction p2 at p1 and p1+1 */
                        int q0[3] = {i, j, k}, q1[3] = {i, j, k};
                        q1[p1] += 1;
                        int64_t i0 = ((int64_t)q0[2] * em[p2][1] + q0[1]) * em[p2][0] + q0[0];
                        int64_t i1 = ((int64_t)q1[2] * em[p2][1] + q1[1]) * em[p2][0] + q1[0];
                        curl = curl + (E[p2][i1] - E[p2][i0]) / g->dx[p1];
                    }
                    if (E[p1]) {   /* - dE_{p1}/dx_{p2} */
                        int q0[3] = {i, j, k}, q1[3] = {i, j, k};
                        q1[p2] += 1;
                        int64_t i0 = ((int64_t)q0[2] * em[p1][1] + q0[1]) * em[p1][0] + q0[0];
                        int64_t i1 = ((int64_t)q1[2] * em[p1][1] + q1[1]) * em[p1][0] + q1[0];
                        curl = curl - (E[p1][i1] - E[p1][i0]) / g->dx[p2];
                    }
                    int64_t f = base + ((int64_t)k * m[1] + j) * m[0] + i;
                    double upd = bs[f] - dt * curl;
                    bout[f] = (stage == 1) ? upd : ca * b0[f] + cb * upd;
                    (void)pos;
                }
    }
    for (int e = 0; e < 3; e++) free(E[e]);
}
