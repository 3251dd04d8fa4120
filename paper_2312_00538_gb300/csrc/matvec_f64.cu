#define ANOVA_REAL double
#include "matvec_prec.inc"
