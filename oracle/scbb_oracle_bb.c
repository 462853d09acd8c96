/* Bounce-back coupling part of the oracle (Sec. II.C-II.E).  Included by scbb_oracle.c. */

static double bb_virtual_psi(osim* s, long n, int x, int y, int z, int i, long m, int c_other,
                             double* react_elem_out, int* elem_out) {
    (void)n; (void)x; (void)y; (void)z; (void)i; (void)react_elem_out; (void)elem_out;
    return psi_of(s, s->rho[c_other * s->N + m]);
}
static void bb_link(osim* s, long n, int x, int y, int z, int i, long m, int c, double fstar, double rho_c) {
    (void)x; (void)y; (void)z; (void)rho_c; (void)n;
    s->fn[(c * s->N + m) * 19 + i] = fstar;
}
static void bb_prepare(osim* s) { (void)s; }
static void bb_after_fluid(osim* s) { (void)s; }
