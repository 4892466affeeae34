// FP32 reduction + refinement route (placeholder until implemented).
#include "common.cuh"
#include "kernels.h"
#include "solver.h"

namespace egb {

int solve_fp32_refine(elsi_gb_handle_s *h, const SolveRequest &rq)
{
    (void)rq;
    return set_error(h, ELSI_ERR_UNSUPPORTED, "FP32_REFINE not available yet");
}

}  // namespace egb
