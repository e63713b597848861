// api.cu -- library and context entry points of libblsh (version, errors,
// context creation, blsh_status).
#include <stdarg.h>

#include "common.cuh"

int blsh_fail(blsh_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int blsh_cuda_check(blsh_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return BLSH_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return blsh_fail(ctx, BLSH_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return blsh_fail(ctx, BLSH_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *blsh_version(void) { return "libblsh 0.1 (sm_103a)"; }

extern "C" const char *blsh_strerror(int code) {
    switch (code) {
    case BLSH_OK: return "ok";
    case BLSH_EINVAL: return "invalid argument";
    case BLSH_ERANGE: return "pair index out of range";
    case BLSH_ETRUNC: return "output truncated";
    case BLSH_ENOMEM: return "out of memory";
    case BLSH_EDEVICE: return "CUDA error";
    case BLSH_ENUMERIC: return "numerical problem in the inference tables";
    case BLSH_ESIZE: return "problem larger than a fixed-size scratch array of the library";
    default: return "unknown error";
    }
}

extern "C" int blsh_ctx_create(blsh_ctx **out, int device) {
    if (!out) return BLSH_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return BLSH_EDEVICE;
    }
    blsh_ctx *ctx = new blsh_ctx();
    ctx->device = device;
    blsh_device_guard g(device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return BLSH_EDEVICE;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->cc_major = prop.major;
    ctx->cc_minor = prop.minor;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    if (prop.major != 10 || prop.minor != 3) {
        // The kernels are compiled for sm_103a only.
        delete ctx;
        return BLSH_EDEVICE;
    }
    if (cudaMalloc((void **)&ctx->scratch, sizeof(blsh_dev_scratch)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return BLSH_ENOMEM;
    }
    if (cudaMalloc((void **)&ctx->recheck_queue, sizeof(uint2) * BLSH_RECHECK_CAP) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->scratch);
        delete ctx;
        return BLSH_ENOMEM;
    }
    if (cudaMemset(ctx->scratch, 0, sizeof(blsh_dev_scratch)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(ctx->scratch);
        cudaFree(ctx->recheck_queue);
        delete ctx;
        return BLSH_EDEVICE;
    }
    *out = ctx;
    return BLSH_OK;
}

extern "C" int blsh_ctx_destroy(blsh_ctx *ctx) {
    if (!ctx) return BLSH_OK;
    {
        blsh_device_guard g(ctx->device);
        if (ctx->scratch) cudaFree(ctx->scratch);
        if (ctx->recheck_queue) cudaFree(ctx->recheck_queue);
    }
    delete ctx;
    return BLSH_OK;
}

extern "C" const char *blsh_last_error(const blsh_ctx *ctx) { return ctx ? ctx->err : "no context"; }

extern "C" int blsh_status(blsh_ctx *ctx, void *stream, uint64_t *counters) {
    if (!ctx) return BLSH_EINVAL;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return blsh_cuda_check(ctx, e, "cudaStreamSynchronize");
    struct {
        unsigned int err_code, pad0;
        unsigned long long counters[4];
    } h;
    BLSH_CUDA(ctx, cudaMemcpyAsync(&h, ctx->scratch, sizeof(h), cudaMemcpyDeviceToHost, s));
    BLSH_CUDA(ctx, cudaMemsetAsync(ctx->scratch, 0, sizeof(h), s));
    BLSH_CUDA(ctx, cudaStreamSynchronize(s));
    if (counters)
        for (int i = 0; i < 4; i++) counters[i] = h.counters[i];
    if (h.err_code == BLSH_ERANGE)
        return blsh_fail(ctx, BLSH_ERANGE, "%llu pairs named an object index >= N", h.counters[0]);
    if (h.err_code == BLSH_ETRUNC)
        return blsh_fail(ctx, BLSH_ETRUNC, "%llu outputs exceeded their capacity", h.counters[1]);
    if (h.err_code != 0) return blsh_fail(ctx, (int)h.err_code, "device error %u", h.err_code);
    return BLSH_OK;
}

extern "C" int64_t blsh_launch_count(const blsh_ctx *ctx) {
    return ctx ? (int64_t)ctx->launches.load(std::memory_order_relaxed) : -1;
}
