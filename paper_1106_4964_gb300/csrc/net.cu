// Learned gauge-covariant preconditioner (no counterpart in the paper).
// State and entry points used by the flexible CG in solver.cu.
#include "ctx.h"

namespace ov {

struct NetState {
    int trained = 0;
};

bool net_ready(const ov_ctx* c) { return c->net && c->net->trained; }

void net_free(ov_ctx* c)
{
    delete c->net;
    c->net = nullptr;
}

int net_apply_precond(ov_ctx* c, const FieldDesc& r, const FieldDesc& z, cudaStream_t st)
{
    (void)r;
    (void)z;
    (void)st;
    return set_err(c, OV_ESTATE, "learned preconditioner not trained");
}

}  // namespace ov
