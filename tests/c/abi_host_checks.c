/* Plain C99 client of the C ABI: host-side argument checks of mrcm_create,
 * which run before any device work, so this program needs no GPU.  Exit
 * status 0 when every case returns the documented code. */
#include <stdio.h>
#include <string.h>

#include "mrcm.h"

/* rc against want; a failing create that returned a handle must carry error
 * text in it (copied before the handle is released). */
static int expect(const char* what, int rc, int want, mrcm_handle* h) {
    char msg[256] = "";
    if (h) {
        const char* m = mrcm_last_error(h);
        if (m) {
            strncpy(msg, m, sizeof msg - 1);
            msg[sizeof msg - 1] = '\0';
        }
        mrcm_destroy(h);
    }
    if (rc != want) {
        fprintf(stderr, "%s: returned %d, expected %d (%s)\n", what, rc, want, msg);
        return 1;
    }
    if (h && want != MRCM_OK && !msg[0]) {
        fprintf(stderr, "%s: no error text\n", what);
        return 1;
    }
    return 0;
}

int main(void) {
    enum { N = 16 };
    static double K[N * N], f[N * N];
    for (int c = 0; c < N * N; ++c) {
        K[c] = 1.0;
        f[c] = 0.0;
    }
    mrcm_grid g;
    memset(&g, 0, sizeof g);
    g.dim = 2;
    g.n[0] = g.n[1] = N;
    g.h[0] = g.h[1] = 1.0 / N;
    mrcm_bc bc;
    memset(&bc, 0, sizeof bc);
    bc.kind[0] = bc.kind[1] = MRCM_DIRICHLET;
    bc.value[0] = 1.0;
    mrcm_partition pt;
    memset(&pt, 0, sizeof pt);
    pt.sub[0] = pt.sub[1] = 8;
    pt.overlap = 2;
    mrcm_params pr;
    memset(&pr, 0, sizeof pr);
    pr.space = MRCM_P1;
    pr.alpha_basis = pr.alpha_smooth = 1.0;
    pr.precision = MRCM_MIXED;
    pr.ir_tol = 1e-12;
    pr.max_ir = 30;
    pr.particular = MRCM_PARTICULAR_OMEGA;

    int bad = 0;
    mrcm_handle* h = NULL;
    mrcm_grid g4 = g;
    g4.dim = 4;
    bad += expect("dim 4", mrcm_create(&g4, K, f, &bc, &pt, &pr, 0, NULL, &h), MRCM_ERR_BAD_INPUT, h);
    h = NULL;
    mrcm_partition p5 = pt;
    p5.sub[0] = 5;
    bad += expect("sub 5 of 16", mrcm_create(&g, K, f, &bc, &p5, &pr, 0, NULL, &h), MRCM_ERR_BAD_INPUT, h);
    h = NULL;
    mrcm_partition p4 = pt;
    p4.overlap = 4;
    bad += expect("overlap 4 of 8", mrcm_create(&g, K, f, &bc, &p4, &pr, 0, NULL, &h), MRCM_ERR_BAD_INPUT, h);
    h = NULL;
    mrcm_params q = pr;
    q.particular = 2;
    bad += expect("particular 2", mrcm_create(&g, K, f, &bc, &pt, &q, 0, NULL, &h), MRCM_ERR_BAD_INPUT, h);
    h = NULL;
    q = pr;
    q.alpha_basis = 0.0;
    bad += expect("alpha 0", mrcm_create(&g, K, f, &bc, &pt, &q, 0, NULL, &h), MRCM_ERR_BAD_INPUT, h);
    h = NULL;
    K[37] = -1.0;
    bad += expect("negative K", mrcm_create(&g, K, f, &bc, &pt, &pr, 0, NULL, &h), MRCM_ERR_BAD_INPUT, h);
    K[37] = 1.0;
    bad += expect("null out", mrcm_create(&g, K, f, &bc, &pt, &pr, 0, NULL, NULL), MRCM_ERR_BAD_INPUT, NULL);
    if (!bad) printf("ok\n");
    return bad ? 1 : 0;
}
