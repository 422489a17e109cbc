// mts.cu -- multi-time-step Arlequin coupling (Sec. 2.5, Alg. 1).
#include "pd.h"

using namespace pdmts;

int mts_time_changed(pdmts_ctx *) { return PDMTS_OK; }

extern "C" int mts_destroy_coupling(pdmts_ctx *) { return PDMTS_OK; }

int mts_advance_coupled(pdmts_ctx *, int64_t)
{
    return fail(PDMTS_ERR_UNSUPPORTED, "mts_advance: coupled stepping not available");
}
