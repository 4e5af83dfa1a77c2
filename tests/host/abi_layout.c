/* Prints, one "name value" pair per line, what a C program sees of
   include/abcmb.h: the size and field offsets of abcmb_options, the status
   codes, the record layout constants and the scalar slots.  Built as strict
   ISO C by tests/test_header_c.py, which compares every line with the
   Python binding's mirror of the same declarations. */
#include <stddef.h>
#include <stdio.h>

#include "abcmb.h"

#define SIZE(t) printf("sizeof.%s %lu\n", #t, (unsigned long)sizeof(t))
#define OFF(f) printf("offset.%s %lu\n", #f, (unsigned long)offsetof(abcmb_options, f))
#define INT(c) printf("%s %ld\n", #c, (long)(c))

int main(void)
{
    SIZE(abcmb_options);
    OFF(lmax_g);
    OFF(lmax_pol);
    OFF(lmax_nu);
    OFF(lmax_cl);
    OFF(n_tau);
    OFF(max_steps);
    OFF(rtol);
    OFF(atol);
    OFF(scale_sw);
    OFF(scale_isw);
    OFF(scale_dop);
    OFF(scale_pol);
    OFF(m_ncdm);
    OFF(lmax_ncdm);
    OFF(node_recipe);
    OFF(n_wide);
    OFF(err_floor);

    INT(ABCMB_OK);
    INT(ABCMB_E_INVALID_ARG);
    INT(ABCMB_E_CUDA);
    INT(ABCMB_E_MAX_STEPS);
    INT(ABCMB_E_NONFINITE);
    INT(ABCMB_E_BACKGROUND);
    INT(ABCMB_E_SCRATCH_TOO_SMALL);
    INT(ABCMB_NPARAM);
    INT(ABCMB_NOALLOC_SCRATCH_BYTES);

    INT(ABCMB_BG_NSCALAR);
    INT(ABCMB_BG_PER_UNIT);
    printf("ABCMB_BG_LNA0 %.17g\n", (double)ABCMB_BG_LNA0);
    INT(ABCMB_BG_NLNA);
    INT(ABCMB_BG_TABLE);
    INT(ABCMB_BG_ODETAB);
    INT(ABCMB_BG_NODES);
    INT(ABCMB_BG_ODEPOLY_DOUBLES);
    INT(ABCMB_BG_LEN(6000));

    INT(ABCMB_S_STATUS);
    INT(ABCMB_S_H0);
    INT(ABCMB_S_OMB);
    INT(ABCMB_S_OMC);
    INT(ABCMB_S_OMG);
    INT(ABCMB_S_OMNU);
    INT(ABCMB_S_OML);
    INT(ABCMB_S_RNU);
    INT(ABCMB_S_FHE);
    INT(ABCMB_S_NH0);
    INT(ABCMB_S_AS);
    INT(ABCMB_S_NS);
    INT(ABCMB_S_ZREION);
    INT(ABCMB_S_LNA_TC);
    INT(ABCMB_S_LNA_SW);
    INT(ABCMB_S_TAU0);
    INT(ABCMB_S_LNA_HE3);
    INT(ABCMB_S_LNA_700);
    INT(ABCMB_S_NTAU);
    INT(ABCMB_S_COUNT);
    return 0;
}
