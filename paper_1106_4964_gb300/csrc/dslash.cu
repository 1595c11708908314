// Wilson dslash launch: validates the launch configuration and hands it to the translation unit
// that holds the chosen variant (the kernels and their layout are described in dslash_common.cuh).
#include "ov_internal.cuh"
#include "ov_kernels.h"

namespace ov {

cudaError_t launch_dslash(const DslashArgs& A, int sp, int gp, int ny, int bx, int by, int var, cudaStream_t st)
{
    if (bx <= 0 || by <= 0 || bx * by > (wide(sp) ? 256 : 512)) return cudaErrorInvalidValue;
    const dim3 block(bx, by);
    // one dimension: 2 parities x site blocks x right-hand-side groups (the kernels' block_work)
    const dim3 grid((unsigned)(2 * ((A.g.Vh + bx - 1) / bx) * ((A.nrhs + by - 1) / by)));
    if (var >= 0 && var <= 2) return launch_dslash_regs(A, sp, gp, ny, var, grid, block, st);
    if (var >= 3 && var <= 5) return launch_dslash_staged(A, sp, gp, ny, var, grid, block, st);
    if (var == 6 || var == 7) return launch_dslash_multi(A, sp, gp, ny, var, grid, block, st);
    if (var == 8 || var == 9) return launch_dslash_batched(A, sp, gp, ny, var, grid, block, st);
    if (var == 10 || var == 11) return launch_dslash_pair(A, sp, gp, ny, var, grid, block, st);
    return cudaErrorInvalidValue;
}

}  // namespace ov
