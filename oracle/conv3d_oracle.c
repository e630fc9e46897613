/*
 * conv3d_oracle.c -- plain FP64 CPU reference of the learned closure's layers.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE (same rules as icarus_oracle.c): only tests/,
 * __graft_entry__.smoke() and bench.py's CPU legs may load it; the CUDA library never does.
 *
 * One layer: y = act(conv3(P(x)) + b), a 3x3x3 cross-correlation over a grid (n1, n2, n3) of
 * C-channel cells, O output channels, where P pads one ghost layer per side: replicate along
 * directions 1 and 2 (r, theta) and circular along direction 3 (phi). act = identity or ReLU.
 * Layout: channels last, x[((k * n2 + j) * n1 + i) * C + c]; weights w[o][tap][c] with
 * tap = (d3 + 1) * 9 + (d2 + 1) * 3 + (d1 + 1) for offsets d in {-1, 0, 1}; bias b[o].
 * Backward: given g = dL/dy, returns dL/dx, dL/dw, dL/db, by the chain rule written out
 * (ReLU mask from y > 0; the padding's adjoint adds each ghost's gradient to the cell it copied).
 */
#include <stdlib.h>
#include <string.h>

static int pad_index(int i, int n, int circular)
{
    if (i < 0) return circular ? i + n : 0;
    if (i >= n) return circular ? i - n : n - 1;
    return i;
}

static long cell(int i, int j, int k, int n1, int n2) { return ((long)k * n2 + j) * n1 + i; }

void orc_conv3d_forward(const double *x, const double *w, const double *b, double *y, int n1, int n2, int n3,
                        int C, int O, int act)
{
#pragma omp parallel for collapse(2)
    for (int k = 0; k < n3; k++)
        for (int j = 0; j < n2; j++)
            for (int i = 0; i < n1; i++)
                for (int o = 0; o < O; o++) {
                    double s = b[o];
                    for (int d3 = -1; d3 <= 1; d3++)
                        for (int d2 = -1; d2 <= 1; d2++)
                            for (int d1 = -1; d1 <= 1; d1++) {
                                int t = (d3 + 1) * 9 + (d2 + 1) * 3 + (d1 + 1);
                                long src = cell(pad_index(i + d1, n1, 0), pad_index(j + d2, n2, 0),
                                                pad_index(k + d3, n3, 1), n1, n2);
                                for (int c = 0; c < C; c++) s += w[((long)o * 27 + t) * C + c] * x[src * C + c];
                            }
                    if (act == 1 && s < 0.0) s = 0.0;
                    y[cell(i, j, k, n1, n2) * O + o] = s;
                }
}

/* g = dL/dy (post-activation); y = forward output (for the ReLU mask) */
void orc_conv3d_backward(const double *x, const double *w, const double *y, const double *g, double *dx,
                         double *dw, double *db, int n1, int n2, int n3, int C, int O, int act)
{
    long N = (long)n1 * n2 * n3;
    double *gp = (double *)malloc(sizeof(double) * N * O);   /* dL/d(pre-activation) */
    for (long q = 0; q < N * O; q++) gp[q] = (act == 1 && !(y[q] > 0.0)) ? 0.0 : g[q];
    memset(dx, 0, sizeof(double) * N * C);
    memset(dw, 0, sizeof(double) * (long)O * 27 * C);
    memset(db, 0, sizeof(double) * O);
    /* straightforward serial accumulation: every (output cell, tap, channel) product once */
    for (int k = 0; k < n3; k++)
        for (int j = 0; j < n2; j++)
            for (int i = 0; i < n1; i++)
                for (int o = 0; o < O; o++) {
                    double go = gp[cell(i, j, k, n1, n2) * O + o];
                    db[o] += go;
                    for (int d3 = -1; d3 <= 1; d3++)
                        for (int d2 = -1; d2 <= 1; d2++)
                            for (int d1 = -1; d1 <= 1; d1++) {
                                int t = (d3 + 1) * 9 + (d2 + 1) * 3 + (d1 + 1);
                                long src = cell(pad_index(i + d1, n1, 0), pad_index(j + d2, n2, 0),
                                                pad_index(k + d3, n3, 1), n1, n2);
                                for (int c = 0; c < C; c++) {
                                    dw[((long)o * 27 + t) * C + c] += go * x[src * C + c];
                                    dx[src * C + c] += go * w[((long)o * 27 + t) * C + c];
                                }
                            }
                }
    free(gp);
}

/* volume-weighted restriction of a fine state [8][2 n3][2 n2][2 n1] onto the coarse grid
 * [8][n3][n2][n1]: U_c = sum_f V_f U_f / sum_f V_f over the 2x2x2 fine cells of each coarse cell;
 * vol_f [2 n3][2 n2][2 n1] are the fine cell volumes */
void orc_restrict(const double *Uf, const double *vol_f, double *Uc, int n1, int n2, int n3)
{
    const int f1 = 2 * n1, f2 = 2 * n2, f3 = 2 * n3;
    const long Nf = (long)f1 * f2 * f3, Nc = (long)n1 * n2 * n3;
    for (int v = 0; v < 8; v++)
        for (int k = 0; k < n3; k++)
            for (int j = 0; j < n2; j++)
                for (int i = 0; i < n1; i++) {
                    double s = 0.0, vs = 0.0;
                    for (int c = 0; c < 8; c++) {
                        int a = 2 * i + (c & 1), bb = 2 * j + ((c >> 1) & 1), cc = 2 * k + ((c >> 2) & 1);
                        long q = ((long)cc * f2 + bb) * f1 + a;
                        s += vol_f[q] * Uf[v * Nf + q];
                        vs += vol_f[q];
                    }
                    Uc[v * Nc + ((long)k * n2 + j) * n1 + i] = s / vs;
                }
}
