// Immutable device copies of small host tables (per-problem launch arguments,
// block offsets), one per distinct content.  A table is written once, before
// its first use, and never changed while it exists, so a captured CUDA graph
// may keep replaying kernels that read it.  Building a table is a synchronous
// copy and must not happen while the stream is being captured.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <unordered_map>
#include <vector>

namespace crl {

class BlobCache {
 public:
  BlobCache() = default;
  BlobCache(const BlobCache&) = delete;
  BlobCache& operator=(const BlobCache&) = delete;
  ~BlobCache() { reset(); }
  // Device copy (256-byte aligned) of `bytes` bytes at `data`; nullptr and
  // *err on failure.
  const void* get(const void* data, size_t bytes, cudaStream_t st, const char** err);
  template <typename T>
  const T* get(const std::vector<T>& v, cudaStream_t st, const char** err) {
    return static_cast<const T*>(get(v.data(), v.size() * sizeof(T), st, err));
  }
  // Frees every table (cudaFree synchronises the device).
  void reset();

 private:
  struct Entry {
    const void* dev;
    std::vector<unsigned char> host;
  };
  std::unordered_map<uint64_t, std::vector<Entry>> map_;
  std::vector<void*> chunks_;
  unsigned char* cur_ = nullptr;
  size_t used_ = 0, cap_ = 0;
};

uint64_t fnv1a64(const void* data, size_t n);

}  // namespace crl
