// K3 in mixed precision (FP32 formal solve). Placeholder until the FP32 kernel lands.
#include "common.cuh"

int mg_launch_feautrier_mixed(mg_ctx *ctx) {
    return mg_fail(ctx, MG_ERR_ARG, "mixed precision formal solve not built yet");
}
