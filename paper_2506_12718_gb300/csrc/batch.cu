// Batched convolutions (pac_convolve_many).
#include "pac_internal.h"

namespace pac {
int run_convolve(pac_plan p, const void* x, void* y, cudaStream_t s);
}

using namespace pac;

extern "C" int pac_convolve_many(int count, const pac_plan* plans, const void* const* x_dev, void* const* y_dev,
                                 void* stream) {
    if (count < 0 || (count > 0 && (!plans || !x_dev || !y_dev))) return fail(PAC_ERR_ARG, "bad arguments");
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !x_dev[i] || !y_dev[i]) return fail(PAC_ERR_ARG, "null entry %d", i);
        if (!plans[i]->has_spec) return fail(PAC_ERR_NO_SPECTRUM, "instance %d: plan has no spectrum", i);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < count; ++i) {
        int rc = run_convolve(plans[i], x_dev[i], y_dev[i], s);
        if (rc) return rc;
    }
    return PAC_OK;
}
