// Allocation-free variant of the operator contraction (pc_apply_operator_static).
//
// pc_apply_operator stages its inputs in the plan's workspace and may grow that
// workspace with cudaMalloc.  Some callers cannot allow that: a caller whose
// device memory is owned by another allocator (a framework's caching pool that
// has reserved the GPU's memory up to a fixed budget), or a latency-sensitive
// caller that must not risk the implicit device synchronisation cudaMalloc and
// cudaFree can cause.  This entry point stages through a fixed array that is
// part of the library image instead, and allocates nothing.
#include "pc_internal.h"

namespace {

// Fixed scratch for the staged operands: 32 MiB, 256-byte aligned.  Every GPU
// that loads the library holds it until the process exits.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device.  In host code
// the array's name is only a host-side stand-in; its device address belongs
// to the current device's context and is looked up, with that device current,
// on every call (a lookup, not an allocation).  It is not cached: after a
// cudaDeviceReset or a new primary context the module is loaded again and the
// address may change.  The first lookup on a device also loads the library's
// device code there, which is why the first call must come before any stream
// capture.
cudaError_t scratch_for_current_device(void **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" pc_status pc_apply_operator_static(pc_plan *p, long long n_ic, const double *x0, const double *g,
                                              double *y, void *stream) {
  if (!p || n_ic < 0 || (n_ic > 0 && (!x0 || !g || !y))) return PC_EINVAL;
  if (n_ic == 0) return PC_OK;
  // staging layout in the fixed array: F [kpad][6][ld], Y [n][6][ld], x0 [6][ld]
  const long long ld = (n_ic + 7) / 8 * 8;
  const size_t rows_f = (size_t)p->kpad * 6, rows_y = (size_t)p->n * 6;
  const size_t need = (rows_f + rows_y + 6) * (size_t)ld * sizeof(double);
  if (ld > (1LL << 30) || need > kStaticScratchBytes) return PC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return PC_EINVAL;
  void *base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess) return PC_ECUDA;
  double *Fs = (double *)base;
  double *Ys = Fs + rows_f * ld;
  double *xs = Ys + rows_y * ld;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t w = (size_t)n_ic * sizeof(double), pitch = (size_t)ld * sizeof(double);
  // The array keeps the previous call's contents: the padding rows of F that
  // the contraction reads must be zeroed for this call's layout.
  e = cudaMemsetAsync(Fs + rows_y * ld, 0, (rows_f - rows_y) * pitch, st);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(xs, pitch, x0, w, w, 6, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(Fs, pitch, g, w, w, rows_y, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = pcx::launch_apply_operator(p, n_ic, (int)ld, xs, Fs, Ys, st);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(y, w, Ys, pitch, w, rows_y, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? PC_OK : PC_ECUDA;
}
