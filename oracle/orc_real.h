/*
 * ORACLE (test infrastructure only; see orc.h).
 *
 * The scalar type of the oracle's arithmetic.  The default build (liborc.so)
 * computes in double.  Built with -DORC_CS (liborc_cs.so) it computes the
 * same statements in double complex, for forward sensitivities by the
 * complex step (Squire & Trapp, SIAM Review 40 (1998) 110; Martins, Sturdza
 * & Alonso, ACM TOMS 29 (2003) 245): with one input set to p + i h, every
 * quantity carries f(p) in its real part and h df/dp in its imaginary part,
 * to rounding, since no difference of nearby values is ever taken.  This is
 * forward-mode differentiation of the whole path (background, thermal
 * history, perturbations, projection, C_ell), the mode the paper's gradients
 * use (Sec. 3).  Branches, table indices, pivots and step counts follow the
 * real parts (RE), so the discrete method differentiated is the one the
 * default build runs; |x| keeps the sign rule of the real part (ABS), which
 * is the analytic continuation away from x = 0; root finds add the first-order
 * correction of their root's imaginary part (orc_background.c).
 */
#ifndef ORC_REAL_H
#define ORC_REAL_H

#ifdef ORC_CS
#include <complex.h>
#include <tgmath.h>
typedef double complex real_t;
#define RE(x) creal(x)
#define IM(x) cimag(x)
static inline real_t orc_abs_cs(real_t x) { return creal(x) < 0.0 ? -x : x; }
#define ABS(x) orc_abs_cs(x)
#define ORC_CS_EXTRA 2 /* further iterations of converged fixed-point solves */
#else
#include <math.h>
typedef double real_t;
#define RE(x) (x)
#define IM(x) (0.0 * (x))
#define ABS(x) fabs(x)
#define ORC_CS_EXTRA 0
#endif

#endif
