#define ANOVA_REAL float
#include "matvec_prec.inc"
