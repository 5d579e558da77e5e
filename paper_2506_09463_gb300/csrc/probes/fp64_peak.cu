// fp64_peak.cu -- measurement probe (not linked into libslqr): throughput of
// the FP64 FMA pipe (DFMA), of FP64 mma.sync (DMMA m8n8k4, m16n8k4, m16n8k16)
// and of FP32 FMA, with register-only kernels timed by CUDA events.  It sets
// the FP64 roofline denominator of the benchmark.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_peak fp64_peak.cu
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("err %s line %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

__global__ void dfma_kernel(double* out, int iters, double a, double b){
  double acc[8];
  #pragma unroll
  for(int i=0;i<8;i++) acc[i]=threadIdx.x*1e-3+i;
  for(int it=0; it<iters; ++it){
    #pragma unroll
    for(int i=0;i<8;i++) acc[i]=fma(acc[i],a,b);
  }
  double s=0;
  #pragma unroll
  for(int i=0;i<8;i++) s+=acc[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
__global__ void ffma_kernel(float* out, int iters, float a, float b){
  float acc[8];
  #pragma unroll
  for(int i=0;i<8;i++) acc[i]=threadIdx.x*1e-3f+i;
  for(int it=0; it<iters; ++it){
    #pragma unroll
    for(int i=0;i<8;i++) acc[i]=fmaf(acc[i],a,b);
  }
  float s=0;
  #pragma unroll
  for(int i=0;i<8;i++) s+=acc[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// m8n8k4 f64: A 1 reg, B 1 reg, C/D 2 regs
__global__ void dmma884_kernel(double* out, int iters){
  double a = 1.0 + threadIdx.x*1e-6, b = 0.5;
  double c[4][2];
  #pragma unroll
  for(int i=0;i<4;i++){c[i][0]=0;c[i][1]=0;}
  for(int it=0; it<iters; ++it){
    #pragma unroll
    for(int i=0;i<4;i++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
        : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
  }
  double s=0;
  #pragma unroll
  for(int i=0;i<4;i++) s+=c[i][0]+c[i][1];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// m16n8k4 f64: A 2 regs, B 1 reg, C/D 4 regs
__global__ void dmma1684_kernel(double* out, int iters){
  double a0 = 1.0 + threadIdx.x*1e-6, a1=0.25, b = 0.5;
  double c[4][4];
  #pragma unroll
  for(int i=0;i<4;i++) for(int j=0;j<4;j++) c[i][j]=0;
  for(int it=0; it<iters; ++it){
    #pragma unroll
    for(int i=0;i<4;i++)
      asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+d"(c[i][0]), "+d"(c[i][1]), "+d"(c[i][2]), "+d"(c[i][3]) : "d"(a0), "d"(a1), "d"(b));
  }
  double s=0;
  #pragma unroll
  for(int i=0;i<4;i++) s+=c[i][0]+c[i][1]+c[i][2]+c[i][3];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// m16n8k16 f64: A 8 regs, B 4 regs, C/D 4 regs
__global__ void dmma16816_kernel(double* out, int iters){
  double a[8], b[4];
  #pragma unroll
  for(int i=0;i<8;i++) a[i]=1.0+threadIdx.x*1e-6+i;
  #pragma unroll
  for(int i=0;i<4;i++) b[i]=0.5+i;
  double c[2][4];
  #pragma unroll
  for(int i=0;i<2;i++) for(int j=0;j<4;j++) c[i][j]=0;
  for(int it=0; it<iters; ++it){
    #pragma unroll
    for(int i=0;i<2;i++)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
        : "+d"(c[i][0]), "+d"(c[i][1]), "+d"(c[i][2]), "+d"(c[i][3])
        : "d"(a[0]),"d"(a[1]),"d"(a[2]),"d"(a[3]),"d"(a[4]),"d"(a[5]),"d"(a[6]),"d"(a[7]),
          "d"(b[0]),"d"(b[1]),"d"(b[2]),"d"(b[3]));
  }
  double s=0;
  #pragma unroll
  for(int i=0;i<2;i++) s+=c[i][0]+c[i][1]+c[i][2]+c[i][3];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}

int main(){
  int dev=0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,dev));
  printf("device %s SMs %d cc %d.%d\n", p.name, p.multiProcessorCount, p.major, p.minor);
  int sms=p.multiProcessorCount;
  const int threads=256; 
  int blocks_list[3]={sms*2, sms*4, sms*8};
  double* out; CK(cudaMalloc(&out, sizeof(double)*sms*8*threads));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for(int bi=0; bi<3; bi++){
    int blocks=blocks_list[bi];
    int iters=4096;
    // DFMA
    for(int rep=0; rep<2; rep++){
      dfma_kernel<<<blocks,threads>>>(out,iters,1.0000001,1e-9); CK(cudaGetLastError());
      cudaEventRecord(e0); dfma_kernel<<<blocks,threads>>>(out,iters,1.0000001,1e-9); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      float ms; cudaEventElapsedTime(&ms,e0,e1);
      double flops=2.0*8*iters*(double)blocks*threads;
      if(rep) printf("DFMA blocks=%d: %.3f ms  %.1f GFLOP/s\n", blocks, ms, flops/ms/1e6);
    }
    for(int rep=0; rep<2; rep++){
      ffma_kernel<<<blocks,threads>>>((float*)out,iters*4,1.0000001f,1e-9f); CK(cudaGetLastError());
      cudaEventRecord(e0); ffma_kernel<<<blocks,threads>>>((float*)out,iters*4,1.0000001f,1e-9f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      float ms; cudaEventElapsedTime(&ms,e0,e1);
      double flops=2.0*8*iters*4*(double)blocks*threads;
      if(rep) printf("FFMA blocks=%d: %.3f ms  %.1f GFLOP/s\n", blocks, ms, flops/ms/1e6);
    }
    for(int rep=0; rep<2; rep++){
      dmma884_kernel<<<blocks,threads>>>(out,iters/4); CK(cudaGetLastError());
      cudaEventRecord(e0); dmma884_kernel<<<blocks,threads>>>(out,iters/4); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      float ms; cudaEventElapsedTime(&ms,e0,e1);
      double flops=2.0*8*8*4*4*(iters/4)*(double)blocks*(threads/32);
      if(rep) printf("DMMA m8n8k4 blocks=%d: %.3f ms  %.1f GFLOP/s\n", blocks, ms, flops/ms/1e6);
    }
    for(int rep=0; rep<2; rep++){
      dmma1684_kernel<<<blocks,threads>>>(out,iters/4); CK(cudaGetLastError());
      cudaEventRecord(e0); dmma1684_kernel<<<blocks,threads>>>(out,iters/4); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      float ms; cudaEventElapsedTime(&ms,e0,e1);
      double flops=2.0*16*8*4*4*(iters/4)*(double)blocks*(threads/32);
      if(rep) printf("DMMA m16n8k4 blocks=%d: %.3f ms  %.1f GFLOP/s\n", blocks, ms, flops/ms/1e6);
    }
    for(int rep=0; rep<2; rep++){
      dmma16816_kernel<<<blocks,threads>>>(out,iters/16); CK(cudaGetLastError());
      cudaEventRecord(e0); dmma16816_kernel<<<blocks,threads>>>(out,iters/16); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
      float ms; cudaEventElapsedTime(&ms,e0,e1);
      double flops=2.0*16*8*16*2*(iters/16)*(double)blocks*(threads/32);
      if(rep) printf("DMMA m16n8k16 blocks=%d: %.3f ms  %.1f GFLOP/s\n", blocks, ms, flops/ms/1e6);
    }
  }
  CK(cudaDeviceSynchronize());
  cudaFree(out);
  return 0;
}
