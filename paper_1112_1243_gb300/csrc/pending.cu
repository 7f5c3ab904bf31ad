// Entry points whose kernels live in later translation units.
#include "dd_internal.h"

extern "C" int dd_logdet_exact(dd_t h, const void*, int, double*) {
    return dd_fail(h, DD_ERR_UNSUPPORTED, "dd_logdet_exact: not built");
}
int block_filter_exact(dd_handle* h, const double*, const double*, int, double*) {
    return dd_fail(h, DD_ERR_UNSUPPORTED, "exact block filter: not built");
}
