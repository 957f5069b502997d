// ski_sketch_hash_noalloc: the hash sketch (no premix) with its bucket-list
// scratch in a fixed device array owned by this library, for callers that
// cannot allocate device memory themselves.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// host callback or another library's stream-ordered region, in a real-time
// loop whose memory was fixed up front, or in a process whose allocator
// belongs to someone else (a framework's caching allocator, a custom pool)
// and which therefore cannot hand this library a workspace pointer.
//
// The scratch is one file-scope __device__ array of SKI_NOALLOC_SCRATCH_BYTES
// (4 MiB); every GPU that loads the library holds it until the process
// exits.  Its device address is looked up on every call, with the caller's
// device current, so it stays right if the context is torn down and created
// again (the module may then load at another address).  The first call on a
// device may load the module there, so that first call should come before
// any stream capture.  All calls share the array: calls that overlap on the
// GPU (different streams, or different host threads on one device) race on
// it and must be serialised by the caller.
#include "common.cuh"
#include "sketch_impl.cuh"

#define SKI_NOALLOC_SCRATCH_BYTES (4u << 20)  // 4 MiB
#define SKI_NOALLOC_MAX_PAIRS 262144          // rows * s
#define SKI_NOALLOC_MAX_M 32768

static __device__ __align__(256) unsigned char g_ski_noalloc_scratch[SKI_NOALLOC_SCRATCH_BYTES];

namespace {
// The array's address on the current device.  In host code the array's name
// is only a host-side stand-in, never a device address.
ski_status scratch_for_current_device(void** out) {
  void* p = nullptr;
  SKI_CUDA_TRY(cudaGetSymbolAddress(&p, g_ski_noalloc_scratch));
  *out = p;
  return SKI_OK;
}
}  // namespace

extern "C" ski_status ski_sketch_hash_noalloc(const ski_matrix* A, const double* b, const ski_opts* o, void* SA,
                                              int64_t ld_sa, void* stream) {
  if (!A || !o || !SA) return SKI_EINVAL;
  if (o->premix || o->hash_kind == 2) return SKI_EINVAL;
  // the s-hashing variant (hash_kind 1) draws with replacement: s may exceed m
  if (A->n < 1 || A->d < 1 || o->s < 1 || o->s > 64 || o->m < (o->hash_kind == 1 ? 1 : o->s)) return SKI_EINVAL;
  if (A->n * (int64_t)o->s > SKI_NOALLOC_MAX_PAIRS || o->m > SKI_NOALLOC_MAX_M) return SKI_EINVAL;
  if (ld_sa < A->d + (b ? 1 : 0)) return SKI_EINVAL;
  const size_t need = ski_sketch_workspace_size(A, b != nullptr, o);
  if (need == 0 || need > SKI_NOALLOC_SCRATCH_BYTES) return SKI_EINVAL;
  void* scratch = nullptr;
  SKI_TRY(scratch_for_current_device(&scratch));
  return ski_sketch_hash(A, b, o, SA, ld_sa, scratch, SKI_NOALLOC_SCRATCH_BYTES, stream);
}
