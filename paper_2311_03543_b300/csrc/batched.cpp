// compar_gemm_batched: many independent GEMMs of uneven sizes in one call.
// Each problem is dispatched through the single-call path (one launch per
// problem, variant chosen per problem).
#include <vector>

#include "runtime.h"

namespace compar {
int gemm_call(compar_ctx* ctx, GemmCall& c, cudaStream_t s);
void batched_release(compar_ctx* ctx) { (void)ctx; }
}  // namespace compar

using namespace compar;

extern "C" int compar_gemm_batched(compar_ctx_t ctx, int count, const compar_problem_t* probs,
                                   double tol, void* stream) {
  if (!ctx || count < 0 || (count > 0 && !probs)) return COMPAR_ERR_INVALID;
  if (ctx->host_only) return COMPAR_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < count; ++i) {
    const compar_problem_t& p = probs[i];
    if (p.m < 0 || p.n < 0 || p.k < 0 || p.lda < p.k || p.ldb < p.n || p.ldc < p.n)
      return COMPAR_ERR_INVALID;
    if (p.dtype != COMPAR_F32 && p.dtype != COMPAR_BF16 && p.dtype != COMPAR_F8E4M3)
      return COMPAR_ERR_INVALID;
    if (p.m > 0 && p.n > 0 && !p.C) return COMPAR_ERR_INVALID;
    if (p.m > 0 && p.n > 0 && p.k > 0 && (!p.A || !p.B)) return COMPAR_ERR_INVALID;
  }
  for (int i = 0; i < count; ++i) {
    const compar_problem_t& p = probs[i];
    GemmCall c;
    c.m = p.m;
    c.n = p.n;
    c.k = p.k;
    c.lda = p.lda;
    c.ldb = p.ldb;
    c.ldc = p.ldc;
    c.dtype = p.dtype;
    c.tol = tol > 0 ? tol : 1e-5;
    c.A = p.A;
    c.B = p.B;
    c.C = p.C;
    c.alpha = p.alpha;
    c.beta = p.beta;
    c.scale_a = p.scale_a;
    c.scale_b = p.scale_b;
    c.batch = count;
    const int rc = gemm_call(ctx, c, s);
    if (rc != COMPAR_OK) return rc;
  }
  return COMPAR_OK;
}
