// PLS decomposition (Eq. (11)-(15)).
#include "dect_internal.cuh"

extern "C" dect_status dect_pls_decompose(const float *, const float *, int, int,
                                          const dect_pls_params *, float *, float *,
                                          dect_pls_report *, dect_stream)
{
    return DECT_ERR_INVALID_ARG;
}
