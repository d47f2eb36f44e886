// Machine-balance probe (not part of libbcg, not compiled by build()): FP64 and FP32 FMA throughput, the
// legacy mma.sync FP64 (m8n8k4) and bf16 (m16n8k16) rates, and HBM copy/read bandwidth, on one GPU with
// CUDA events. Independent FMA chains (8 per thread, 152 x 8 CTAs of 256 threads) keep the pipes full; the
// copy and read loops stream two 1 GiB arrays. Its FP64 : FP32 ratio is what places every FP64 kernel of
// the solver on the FP64-pipe side of the roofline.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 paper_1912_11930_gb300/csrc/peaks_probe.cu -o peaks && ./peaks
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s line %d: %s\n",#x,__LINE__,cudaGetErrorString(e)); return 1;}}while(0)

template<typename T> __global__ void fma_kernel(T* out, int iters, T b, T c) {
  T a0=threadIdx.x, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  for (int i=0;i<iters;i++){
#pragma unroll
    for(int u=0;u<4;u++){
    a0=a0*b+c; a1=a1*b+c; a2=a2*b+c; a3=a3*b+c; a4=a4*b+c; a5=a5*b+c; a6=a6*b+c; a7=a7*b+c;}
  }
  out[blockIdx.x*blockDim.x+threadIdx.x] = a0+a1+a2+a3+a4+a5+a6+a7;
}

__global__ void dmma_kernel(double* out, int iters) {
  double a = threadIdx.x*1e-3, b = 1.0 + threadIdx.x*1e-4;
  double d[4][2];
  for(int s=0;s<4;s++){d[s][0]=0;d[s][1]=0;}
  for (int i=0;i<iters;i++){
#pragma unroll
    for(int s=0;s<4;s++){
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
        : "+d"(d[s][0]), "+d"(d[s][1]) : "d"(a), "d"(b));
    }
  }
  double acc=0; for(int s=0;s<4;s++) acc += d[s][0]+d[s][1];
  out[blockIdx.x*blockDim.x+threadIdx.x] = acc;
}

__global__ void bmma_kernel(float* out, int iters) {
  uint32_t a[4], b[2];
  for(int i=0;i<4;i++) a[i] = 0x3f803f80u ^ (threadIdx.x<<3);
  for(int i=0;i<2;i++) b[i] = 0x3f803f80u;
  float d[4][4];
  for(int s=0;s<4;s++) for(int j=0;j<4;j++) d[s][j]=0.f;
  for (int i=0;i<iters;i++){
#pragma unroll
    for(int s=0;s<4;s++){
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[s][0]), "+f"(d[s][1]), "+f"(d[s][2]), "+f"(d[s][3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
  }
  float acc=0; for(int s=0;s<4;s++) for(int j=0;j<4;j++) acc += d[s][j];
  out[blockIdx.x*blockDim.x+threadIdx.x] = acc;
}

__global__ void copy_kernel(const double2* __restrict__ a, double2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x*(size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x*blockDim.x) b[i] = a[i];
}
__global__ void read_kernel(const double2* __restrict__ a, double* out, size_t n) {
  double s = 0;
  for (size_t i = blockIdx.x*(size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x*blockDim.x) { double2 v = a[i]; s += v.x + v.y; }
  if (s == 12345.678) out[0] = s;
}

int main() {
  int dev=0; cudaDeviceProp pr; CK(cudaGetDeviceProperties(&pr, dev));
  printf("device %s SMs %d cc %d.%d l2 %d MB\n", pr.name, pr.multiProcessorCount, pr.major, pr.minor, pr.l2CacheSize>>20);
  int sms = pr.multiProcessorCount;
  const int threads = 256; const int blocks = sms * 8;
  size_t nthr = (size_t)threads*blocks;
  double* dout; float* fout; CK(cudaMalloc(&dout, nthr*sizeof(double))); CK(cudaMalloc(&fout, nthr*sizeof(float)));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  // FP64 FMA
  for (int rep=0; rep<2; rep++) {
    int it = 2000;
    cudaEventRecord(e0); fma_kernel<double><<<blocks,threads>>>(dout, it, 0.999999, 1e-7); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    double fl = 2.0*32*it*(double)nthr; printf("DFMA: %.3f ms  %.3f TFLOP/s\n", ms, fl/ms/1e9);
  }
  for (int rep=0; rep<2; rep++) {
    int it = 20000;
    cudaEventRecord(e0); fma_kernel<float><<<blocks,threads>>>(fout, it, 0.999999f, 1e-7f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    double fl = 2.0*32*it*(double)nthr; printf("FFMA: %.3f ms  %.3f TFLOP/s\n", ms, fl/ms/1e9);
  }
  for (int rep=0; rep<2; rep++) {
    int it = 500;
    cudaEventRecord(e0); dmma_kernel<<<blocks,threads>>>(dout, it); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    double fl = 512.0*4*it*(double)(nthr/32); printf("DMMA m8n8k4: %.3f ms  %.3f TFLOP/s\n", ms, fl/ms/1e9);
  }
  for (int rep=0; rep<2; rep++) {
    int it = 5000;
    cudaEventRecord(e0); bmma_kernel<<<blocks,threads>>>(fout, it); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    double fl = 4096.0*4*it*(double)(nthr/32); printf("mma.sync bf16 m16n8k16: %.3f ms  %.3f TFLOP/s\n", ms, fl/ms/1e9);
  }
  // HBM: 1 GiB per array
  size_t n2 = (size_t)1<<26; // double2 elements -> 1 GiB
  double2 *a, *b; CK(cudaMalloc(&a, n2*sizeof(double2))); CK(cudaMalloc(&b, n2*sizeof(double2)));
  CK(cudaMemset(a, 0, n2*sizeof(double2)));
  for (int g : {sms*4, sms*8, sms*16}) {
    for (int rep=0; rep<3; rep++) {
      cudaEventRecord(e0); copy_kernel<<<g, 512>>>(a, b, n2); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep==2) printf("copy grid %d: %.3f ms %.1f GB/s\n", g, ms, 2.0*n2*16/ms/1e6);
    }
    for (int rep=0; rep<3; rep++) {
      cudaEventRecord(e0); read_kernel<<<g, 512>>>(a, dout, n2); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep==2) printf("read grid %d: %.3f ms %.1f GB/s\n", g, ms, 1.0*n2*16/ms/1e6);
    }
  }
  CK(cudaGetLastError());
  printf("probe done\n");
  return 0;
}
