// Wilson dslash, launch variants 0-2: one site and one right-hand side per thread, register budgets.
#include "dslash_common.cuh"

namespace ov {

namespace {

template <int SP, int GP, int VAR>
cudaError_t launch_var(const DslashArgs& A, int ny, dim3 grid, dim3 block, cudaStream_t st)
{
    if ((int)(block.x * block.y) > Bounds<SP, VAR>::maxt) return cudaErrorInvalidValue;
    switch (ny) {
    case 0: dslash_kernel<SP, GP, 0, VAR><<<grid, block, 0, st>>>(A); break;
    case 1: dslash_kernel<SP, GP, 1, VAR><<<grid, block, 0, st>>>(A); break;
    case 2: dslash_kernel<SP, GP, 2, VAR><<<grid, block, 0, st>>>(A); break;
    case 3: dslash_kernel<SP, GP, 3, VAR><<<grid, block, 0, st>>>(A); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

struct Regs {
    template <int SP, int GP>
    static cudaError_t run(const DslashArgs& A, int ny, int var, dim3 grid, dim3 block, cudaStream_t st)
    {
        switch (var) {
        case 0: return launch_var<SP, GP, 0>(A, ny, grid, block, st);
        case 1: return launch_var<SP, GP, 1>(A, ny, grid, block, st);
        case 2: return launch_var<SP, GP, 2>(A, ny, grid, block, st);
        }
        return cudaErrorInvalidValue;
    }
};

}  // namespace

cudaError_t launch_dslash_regs(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block, cudaStream_t st)
{
    return dispatch_prec<Regs>(A, sp, gp, ny, var, grid, block, st);
}

}  // namespace ov
