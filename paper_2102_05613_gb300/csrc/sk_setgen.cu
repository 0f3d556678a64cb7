// sk_setgen.cu -- generation probabilities of sets of configurations
// (App. D.1, D.2): Pt(M) = P_gen(S | S \ M) for every subset M of an
// n-element set S, where the set grows by adding one element at a time,
// generated from a parent chosen uniformly in the current set.
//
// The recursion on the first addition,
//   Pt(M) = (1/|S \ M|) sum_{e in M} c(M, e) Pt(M \ {e}),
//   c(M, e) = sum_{p in S \ M} P_gen(e | p),
// needs only subsets with one element fewer, so the masks are processed one
// cardinality at a time, one thread per mask; a thread finds its mask by
// unranking its index in the combinatorial number system.  Two forms:
// direct (each c(M, e) summed afresh, O(n^2 2^n)) and the paper's cumulative
// form (Eq. eq_rec_set_short: c(M, e) = c(M \ {f}, e) - P_gen(e | f) from
// the previous cardinality's table, f the lowest other element of M;
// O(n 2^n) work and a table of n 2^n doubles).  Double precision (the values
// are products of up to n-1 probabilities).
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "sk_internal.h"
#include "sk_mcmcmc.h"

namespace sk {
namespace {

constexpr uint32_t kMaxSetN = 28;

__global__ void setgen_level(const double* __restrict__ Pg, const unsigned long long* __restrict__ binom, uint32_t n,
                             uint32_t m, unsigned long long count, double* __restrict__ out) {
    __shared__ double P[kMaxSetN * kMaxSetN];
    __shared__ unsigned long long C[(kMaxSetN + 1) * (kMaxSetN + 1)];
    for (uint32_t i = threadIdx.x; i < n * n; i += blockDim.x) P[i] = Pg[i];
    for (uint32_t i = threadIdx.x; i < (n + 1) * (n + 1); i += blockDim.x) C[i] = binom[i];
    __syncthreads();
    const unsigned long long idx = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x;
    if (idx >= count) return;
    // the idx-th m-subset in colexicographic order
    uint32_t M = 0;
    unsigned long long r = idx;
    uint32_t left = m;
    for (int b = static_cast<int>(n) - 1; b >= 0 && left; --b) {
        const unsigned long long c = C[b * (n + 1) + left];  // binom(b, left)
        if (c <= r) {
            M |= 1u << b;
            r -= c;
            --left;
        }
    }
    const uint32_t all = (n == 32u) ? 0xFFFFFFFFu : ((1u << n) - 1u);
    const uint32_t cur = all & ~M;
    double tot = 0.0;
    for (uint32_t e = 0; e < n; ++e) {
        if (!((M >> e) & 1u)) continue;
        double a = 0.0;
        for (uint32_t p = 0; p < n; ++p)
            if ((cur >> p) & 1u) a += P[e * n + p];
        tot = fma(a, out[M & ~(1u << e)], tot);
    }
    out[M] = tot / static_cast<double>(n - m);
}

// The cumulative form: as setgen_level, with c(M, e) kept at c[M n + e].
__global__ void setgen_level_cum(const double* __restrict__ Pg, const unsigned long long* __restrict__ binom,
                                 uint32_t n, uint32_t m, unsigned long long count, double* __restrict__ out,
                                 double* __restrict__ c) {
    __shared__ double P[kMaxSetN * kMaxSetN];
    __shared__ unsigned long long C[(kMaxSetN + 1) * (kMaxSetN + 1)];
    for (uint32_t i = threadIdx.x; i < n * n; i += blockDim.x) P[i] = Pg[i];
    for (uint32_t i = threadIdx.x; i < (n + 1) * (n + 1); i += blockDim.x) C[i] = binom[i];
    __syncthreads();
    const unsigned long long idx = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x;
    if (idx >= count) return;
    uint32_t M = 0;
    unsigned long long r = idx;
    uint32_t left = m;
    for (int b = static_cast<int>(n) - 1; b >= 0 && left; --b) {
        const unsigned long long cb = C[b * (n + 1) + left];  // binom(b, left)
        if (cb <= r) {
            M |= 1u << b;
            r -= cb;
            --left;
        }
    }
    double tot = 0.0;
    for (uint32_t e = 0; e < n; ++e) {
        if (!((M >> e) & 1u)) continue;
        const uint32_t rest = M & ~(1u << e);
        double ce;
        if (!rest) {  // c({e}, e): every other element is a parent
            ce = 0.0;
            for (uint32_t p = 0; p < n; ++p)
                if (p != e) ce += P[e * n + p];
        } else {
            const uint32_t f = static_cast<uint32_t>(__ffs(rest) - 1);
            ce = c[static_cast<size_t>(M & ~(1u << f)) * n + e] - P[e * n + f];
        }
        c[static_cast<size_t>(M) * n + e] = ce;
        tot = fma(ce, out[rest], tot);
    }
    out[M] = tot / static_cast<double>(n - m);
}

__global__ void setgen_ends(double* out, uint32_t all) {
    if (threadIdx.x == 0) {
        out[0] = 1.0;
        out[all] = 0.0;
    }
}

}  // namespace
}  // namespace sk

extern "C" sk_status sk_set_generation(uint32_t n, const double* P, double* out, uint32_t mem, uint32_t method,
                                       void* stream) {
    if (!P || !out) {
        sk::set_error_message("sk_set_generation: NULL argument");
        return SK_ERR_INVALID_ARG;
    }
    if (n < 1 || n > sk::kMaxSetN) {
        sk::set_error_message("sk_set_generation: n must be 1..28");
        return SK_ERR_INVALID_ARG;
    }
    if (mem != SK_MEM_HOST && mem != SK_MEM_DEVICE) {
        sk::set_error_message("sk_set_generation: mem must be SK_MEM_HOST or SK_MEM_DEVICE");
        return SK_ERR_INVALID_ARG;
    }
    if (method > SK_SETGEN_CUMULATIVE) {
        sk::set_error_message("sk_set_generation: method must be SK_SETGEN_AUTO, _DIRECT or _CUMULATIVE");
        return SK_ERR_INVALID_ARG;
    }
    for (uint32_t i = 0; i < n * n; ++i)
        if (!(P[i] >= 0.0) || P[i] == INFINITY) {
            sk::set_error_message("sk_set_generation: P must be finite and >= 0");
            return SK_ERR_INVALID_ARG;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nmask = static_cast<size_t>(1) << n;
    std::vector<unsigned long long> C((n + 1) * (n + 1), 0ull);
    for (uint32_t a = 0; a <= n; ++a) {
        C[a * (n + 1)] = 1;
        for (uint32_t b = 1; b <= a; ++b) C[a * (n + 1) + b] = C[(a - 1) * (n + 1) + b - 1] + (b < a ? C[(a - 1) * (n + 1) + b] : 0);
    }
    double* dP = nullptr;
    unsigned long long* dC = nullptr;
    double* dc = nullptr;  // the cumulative table, n 2^n doubles
    double* dout = mem == SK_MEM_DEVICE ? out : nullptr;
    cudaError_t e = cudaSuccess;
    if (method != SK_SETGEN_DIRECT && n > 1) {
        e = cudaMalloc(&dc, nmask * n * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            dc = nullptr;
            if (method == SK_SETGEN_CUMULATIVE) {
                sk::set_error_message("sk_set_generation: no room for the cumulative table (n 2^n doubles)");
                return SK_ERR_OOM;
            }
            e = cudaSuccess;  // auto: the direct form
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&dP, n * n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dC, C.size() * sizeof(unsigned long long));
    if (e == cudaSuccess && !dout) e = cudaMalloc(&dout, nmask * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dP, P, n * n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dC, C.data(), C.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        sk::setgen_ends<<<1, 32, 0, st>>>(dout, static_cast<uint32_t>(nmask - 1));
        e = cudaGetLastError();
    }
    for (uint32_t m = 1; m < n && e == cudaSuccess; ++m) {
        const unsigned long long count = C[n * (n + 1) + m];
        const unsigned long long blocks = (count + 255) / 256;
        if (dc)
            sk::setgen_level_cum<<<static_cast<unsigned>(blocks), 256, 0, st>>>(dP, dC, n, m, count, dout, dc);
        else
            sk::setgen_level<<<static_cast<unsigned>(blocks), 256, 0, st>>>(dP, dC, n, m, count, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && mem == SK_MEM_HOST)
        e = cudaMemcpyAsync(out, dout, nmask * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dP);
    cudaFree(dC);
    cudaFree(dc);
    if (mem == SK_MEM_HOST) cudaFree(dout);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sk::set_error_message(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SK_ERR_OOM : SK_ERR_CUDA;
    }
    return SK_OK;
}
