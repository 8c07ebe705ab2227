// Immutable device tables (see tables.h).
#include <string.h>

#include <algorithm>

#include "tables.h"

namespace crl {

uint64_t fnv1a64(const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

const void* BlobCache::get(const void* data, size_t bytes, cudaStream_t st, const char** err) {
  const uint64_t h = fnv1a64(data, bytes);
  auto it = map_.find(h);
  if (it != map_.end()) {
    for (const Entry& e : it->second)
      if (e.host.size() == bytes && memcmp(e.host.data(), data, bytes) == 0) return e.dev;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    *err = "a launch table was first needed while the stream was being captured";
    return nullptr;
  }
  const size_t need = (bytes + 255) / 256 * 256;
  if (used_ + need > cap_) {
    const size_t cap = std::max<size_t>(need, size_t(1) << 20);
    void* mem = nullptr;
    if (cudaMalloc(&mem, cap) != cudaSuccess) {
      *err = "device allocation of a launch table failed";
      return nullptr;
    }
    chunks_.push_back(mem);
    cur_ = static_cast<unsigned char*>(mem);
    used_ = 0;
    cap_ = cap;
  }
  unsigned char* dev = cur_ + used_;
  if (cudaMemcpy(dev, data, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    *err = "copying a launch table failed";
    return nullptr;
  }
  used_ += need;
  Entry e{dev, std::vector<unsigned char>(static_cast<const unsigned char*>(data),
                                          static_cast<const unsigned char*>(data) + bytes)};
  map_[h].push_back(std::move(e));
  return dev;
}

void BlobCache::reset() {
  for (void* p : chunks_) cudaFree(p);
  chunks_.clear();
  map_.clear();
  cur_ = nullptr;
  used_ = cap_ = 0;
}

}  // namespace crl
