/* CPU oracle for the connected-sum hot path of CoS++ (arXiv 2507.12349).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the timed CPU
 * baseline of the benchmark may load this library; the CUDA product path
 * never does, and shares no code, header or table with it.
 *
 * Three tiers, each in double, long double and __float128 (suffixes _d, _ld,
 * _q; results returned as a double pair hi + lo):
 *   brute   decorated covers enumerated one by one (n <= 5 in practice)
 *   closed  determinants + the subset subtraction of Methods A
 *   dp      the merged clow-sequence DP of Results A / Alg. 2-3, plain loops
 * the bipartite (two-sublattice) sums of oracle_bip.h: the definition (sum over
 * sublattice assignments) and the sublattice-resolved merged DP of Alg. 1-2; and the SU(2)
 * determinant-weight DP without cycle factors of oracle_det.h (Alg. 1).
 * Every function states the passage it follows in oracle_impl.h / oracle_bip.h /
 * oracle_det.h.
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <quadmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define REAL double
#define FN(x) x##_d
#define RABS(x) fabs(x)
#include "oracle_impl.h"
#include "oracle_bip.h"
#include "oracle_det.h"
#undef REAL
#undef FN
#undef RABS

#define REAL long double
#define FN(x) x##_ld
#define RABS(x) fabsl(x)
#include "oracle_impl.h"
#include "oracle_bip.h"
#include "oracle_det.h"
#undef REAL
#undef FN
#undef RABS

#define REAL __float128
#define FN(x) x##_q
#define RABS(x) fabsq(x)
#include "oracle_impl.h"
#include "oracle_bip.h"
#include "oracle_det.h"
#undef REAL
#undef FN
#undef RABS
