// Instruction-throughput microbenchmarks (pipes.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace mcd {

// 8 blocks of 256 threads per SM; per block the SM id and the cycle counter
// at the start and end of its timed loop.
constexpr int kPipeThreads = 256;
constexpr int kPipeBlocksPerSM = 8;
struct PipeKeys {
    uint32_t rk0[10];
    uint32_t rk1[10];
};
// Operations of the measured class per thread and loop step.
int pipe_ops_per_step(int op);
cudaError_t launch_pipe(int op, int iters, int blocks, uint32_t m, float c, uint32_t* sink, long long* t0,
                        long long* t1, int* smid, cudaStream_t s);

}  // namespace mcd
