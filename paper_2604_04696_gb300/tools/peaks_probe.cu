// Peak-rate probes for the RowSel rooflines on this GPU: INT8 mma.sync (IMMA),
// bf16 mma.sync (HMMA), IMAD.WIDE.U32 and IMAD issue rates, L2 read bandwidth,
// and DRAM read bandwidth for p-major rows read in chunks of T consecutive
// slots. Built and run by `python bench.py --peaks`; prints plain text.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d: %s\n", #x, __LINE__, cudaGetErrorString(e)); return 1; } } while (0)

__global__ void imma_peak(int iters, int* out) {
  unsigned a0 = threadIdx.x, a1 = threadIdx.x * 3u, a2 = threadIdx.x * 5u, a3 = threadIdx.x * 7u;
  unsigned b0 = threadIdx.x * 11u, b1 = threadIdx.x * 13u;
  int c[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) { c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                   : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
  int s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
  if (s == 0x7fffffff) out[0] = s;
}

__global__ void hmma_peak(int iters, float* out) {
  unsigned a0 = 0x3f803f80u, a1 = a0, a2 = a0, a3 = a0, b0 = 0x3f803f80u, b1 = b0;
  float c[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) { c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
                   : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
  float s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
  if (s == 1.2345f) out[0] = s;
}

__global__ void imad_wide_peak(int iters, unsigned long long* out) {
  unsigned a[4], b[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) { a[j] = threadIdx.x * (j + 3) + 1; b[j] = blockIdx.x * (j + 5) + 7; }
  unsigned long long c[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) c[j] = j;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(c[j]) : "r"(a[j & 3]), "r"(b[j >> 2]));
    }
  }
  unsigned long long s = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) s ^= c[j];
  if (s == 12345ull) out[0] = s;
}

__global__ void imad_lo_peak(int iters, unsigned* out) {
  unsigned a[4], b[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) { a[j] = threadIdx.x * (j + 3) + 1; b[j] = blockIdx.x * (j + 5) + 7; }
  unsigned c[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) c[j] = j;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(c[j]) : "r"(a[j & 3]), "r"(b[j >> 2]));
    }
  }
  unsigned s = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) s ^= c[j];
  if (s == 12345u) out[0] = s;
}

// Read `n16` uint4 elements `reps` times (grid-stride). Working set small enough to sit in L2.
__global__ void read_rep(const uint4* __restrict__ p, size_t n16, int reps, unsigned* out) {
  unsigned acc = 0;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
      uint4 v = __ldcg(p + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  if (acc == 0x12345678u) out[0] = acc;
}

// Chunked-row read: buffer is rows x row_words uint32. CTA b reads words [b*T, b*T+T) of every row,
// with uint4 loads (T multiple of 4). Rows are walked in order by all CTAs.
__global__ void chunk_read(const uint32_t* __restrict__ p, int rows, int row_words, int T, unsigned* out) {
  int tpr = T / 4;                 // threads per row
  int rows_per_pass = blockDim.x / tpr;
  int tr = threadIdx.x / tpr, tc = threadIdx.x % tpr;
  const uint32_t* base = p + (size_t)blockIdx.x * T + tc * 4;
  unsigned acc = 0;
  for (int r = tr; r < rows; r += rows_per_pass) {
    uint4 v = __ldcs(reinterpret_cast<const uint4*>(base + (size_t)r * row_words));
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x12345678u) out[0] = acc;
}

int main() {
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, 0));
  printf("device %s sms %d l2 %d smem/sm %zu smem/block-optin %zu clock(kHz) %d mem %zu MiB\n", prop.name,
         prop.multiProcessorCount, prop.l2CacheSize, prop.sharedMemPerMultiprocessor, prop.sharedMemPerBlockOptin,
         0, prop.totalGlobalMem >> 20);
  int sms = prop.multiProcessorCount;
  int* dout; CK(cudaMalloc(&dout, 64));
  cudaEvent_t e0, e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  float ms;
  for (int wpb : {4, 8, 16}) {
    int iters = 4096, grid = sms * 4, block = 32 * wpb;
    imma_peak<<<grid, block>>>(16, dout); CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(e0)); imma_peak<<<grid, block>>>(iters, dout); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    double ops = (double)grid * wpb * iters * 8 * 2.0 * 16 * 8 * 32;
    printf("IMMA u8 m16n8k32 warps/blk %d: %.1f TOPS (%.3f ms)\n", wpb, ops / ms / 1e9, ms);
    hmma_peak<<<grid, block>>>(16, (float*)dout); CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(e0)); hmma_peak<<<grid, block>>>(iters, (float*)dout); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ops = (double)grid * wpb * iters * 8 * 2.0 * 16 * 8 * 16;
    printf("HMMA bf16 m16n8k16 warps/blk %d: %.1f TFLOPS (%.3f ms)\n", wpb, ops / ms / 1e9, ms);
  }
  for (int tpb : {256, 512}) {
    int iters = 2048, grid = sms * 4;
    imad_wide_peak<<<grid, tpb>>>(16, (unsigned long long*)dout); CK(cudaGetLastError()); CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(e0)); imad_wide_peak<<<grid, tpb>>>(iters, (unsigned long long*)dout); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    double macs = (double)grid * tpb * iters * 16;
    printf("mad.wide.u32 tpb %d: %.2f T MAC/s (%.3f ms)\n", tpb, macs / ms / 1e9, ms);
    imad_lo_peak<<<grid, tpb>>>(16, (unsigned*)dout); CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(e0)); imad_lo_peak<<<grid, tpb>>>(iters, (unsigned*)dout); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    printf("mad.lo.u32 tpb %d: %.2f T op/s (%.3f ms)\n", tpb, macs / ms / 1e9, ms);
  }
  // L2 read bandwidth
  {
    size_t bytes = 48ull << 20; uint4* buf; CK(cudaMalloc(&buf, bytes)); CK(cudaMemset(buf, 1, bytes));
    size_t n16 = bytes / 16; int reps = 20;
    for (int grid : {sms * 4, sms * 8}) {
      read_rep<<<grid, 512>>>(buf, n16, 2, (unsigned*)dout); CK(cudaDeviceSynchronize());
      CK(cudaEventRecord(e0)); read_rep<<<grid, 512>>>(buf, n16, reps, (unsigned*)dout); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms, e0, e1));
      printf("L2 read (48 MiB x %d) grid %d: %.1f GB/s\n", reps, grid, (double)bytes * reps / ms / 1e6);
    }
    CK(cudaFree(buf));
  }
  // DRAM chunked read: rows of 32 KiB (8192 words), 4 GiB total
  {
    int row_words = 8192; int rows = 131072; size_t bytes = (size_t)rows * row_words * 4;
    uint32_t* buf; CK(cudaMalloc(&buf, bytes)); CK(cudaMemset(buf, 3, bytes));
    for (int T : {4, 8, 16, 32, 64, 128}) {
      int grid = row_words / T;
      for (int block : {256, 1024}) {
        if (block < T / 4) continue;
        chunk_read<<<grid, block>>>(buf, rows, row_words, T, (unsigned*)dout); CK(cudaDeviceSynchronize());
        CK(cudaEventRecord(e0)); chunk_read<<<grid, block>>>(buf, rows, row_words, T, (unsigned*)dout); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        printf("DRAM chunk-read T=%d slots (%d B) block %d grid %d: %.1f GB/s\n", T, T * 4, block, grid, (double)bytes / ms / 1e6);
      }
    }
    // contiguous read for reference
    for (int grid : {sms * 4, sms * 8}) {
      read_rep<<<grid, 512>>>((const uint4*)buf, bytes / 16, 1, (unsigned*)dout); CK(cudaDeviceSynchronize());
      CK(cudaEventRecord(e0)); read_rep<<<grid, 512>>>((const uint4*)buf, bytes / 16, 1, (unsigned*)dout); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms, e0, e1));
      printf("DRAM contiguous read 4 GiB grid %d: %.1f GB/s\n", grid, (double)bytes / ms / 1e6);
    }
    CK(cudaFree(buf));
  }
  printf("done\n");
  return 0;
}
