// Workspace sizing and status helpers shared across translation units.
#pragma once
#include "vr_internal.cuh"

namespace vr {
size_t ws_fof3d(int64_t n);
size_t ws_substructure(int64_t n, const vr_params *p);
vr_status check_ws(vr_ctx *ctx, const Arena &ar, size_t ws_bytes);
vr_status read_status(vr_ctx *ctx, cudaStream_t s, DevStatus *out);
}  // namespace vr
