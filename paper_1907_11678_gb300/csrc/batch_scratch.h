// batch_scratch.h -- size of the batched search's scratch area, shared by the workspace entry
// point (seis_batch_workspace_size) and the allocation-free one, whose fixed array must hold
// exactly what the former asks of a caller.
#pragma once
#include <cstddef>
#include <cstdint>

namespace seis {

// Bytes of batch scratch for n items: the work counter in [0, 256), then the task table of
// n + 1 int64 entries rounded up to 256 bytes.
constexpr size_t batch_workspace_bytes(int64_t n) {
    return n < 0 ? 0 : 256 + ((((size_t)n + 1) * sizeof(int64_t) + 255) & ~(size_t)255);
}

}  // namespace seis
