// Failure detection without a GPU fault: the bounded mbarrier wait that every tensor-core
// pipeline stage uses (tc::mbar_wait) run against a barrier that nothing completes.
//
//   mode 0: nothing arrives and nothing aborts -> the wait gives up after its limit (2 s)
//   mode 1: a second warp raises the abort flag after 20 ms -> the wait gives up then
//   mode 2: the barrier's one arrival happens first -> the wait succeeds at once
//
// Every loop here ends by the global timer; the kernel returns normally in every mode and
// writes {wait succeeded, elapsed ms}, so the context stays usable.
#include "common.cuh"
#include "knn.cuh"
#include "tc_common.cuh"

namespace ssg {

__global__ void k_wait_selftest(int mode, int* __restrict__ out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar), 1);
    abort_flag = 0;
    tc::fence_barrier_init();
  }
  __syncthreads();
  if (mode == 1 && threadIdx.x == 32) {
    const uint64_t t0 = tc::global_ns();
    while (tc::global_ns() - t0 < 20000000ull) {
    }
    *(volatile int*)&abort_flag = 1;
  }
  if (threadIdx.x == 0) {
    if (mode == 2) tc::mbar_arrive(tc::smem_u32(&bar));
    const uint64_t t0 = tc::global_ns();
    const bool ok = tc::mbar_wait(tc::smem_u32(&bar), 0, &abort_flag);
    out[0] = ok ? 1 : 0;
    out[1] = (int)((tc::global_ns() - t0) / 1000000ull);
  }
}

void wait_selftest(int mode, int* ok_host, int* elapsed_ms_host, cudaStream_t st) {
  Scratch<int> out(2, st);
  SSG_LAUNCH(k_wait_selftest, 1, 64, 0, st, mode, out.p);
  int h[2] = {0, 0};
  SSG_CUDA(cudaMemcpyAsync(h, out.p, sizeof(h), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  *ok_host = h[0];
  *elapsed_ms_host = h[1];
}

}  // namespace ssg
