// srp_dense.cu -- sign random projections of dense rows (Section 4.2, "LSH
// family"): bit j of row i = [x_i . r_j >= 0].
#include "common.cuh"

int blsh_srp_dense_simt(blsh_ctx *ctx, const float *X, int64_t N, int32_t d, const float *R, int32_t bits,
                        uint32_t *sig, cudaStream_t s);

extern "C" int blsh_srp_dense(blsh_ctx *ctx, const float *X, int64_t N, int32_t d, const float *R, int32_t bits,
                              float margin, uint32_t *sig, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (!X || !R || !sig) return blsh_fail(ctx, BLSH_EINVAL, "X, R and sig are required");
    if (N < 0 || d <= 0 || bits <= 0 || bits % 32 || bits > 4096 || !(margin >= 0.0f))
        return blsh_fail(ctx, BLSH_EINVAL, "bad N, d, bits or margin");
    if (N == 0) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    return blsh_srp_dense_simt(ctx, X, N, d, R, bits, sig, blsh_stream(stream));
}
