// Throughput probe of the arithmetic and barrier figures the kernels are sized against: FP64, FP32 and
// packed FP32x2 FMA rates, __sincosf rate, device-wide barrier latency (bounded spin), the latency
// of dependent FP64 operations, D2D copy.
// Built and run by paper_1912_10596_gb300/probe.py (a standalone executable, not part of libxflat).
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s line %d: %s\n",#x,__LINE__,cudaGetErrorString(e)); return 1;}}while(0)

__global__ void fma64(double* out, int iters, double s){
  double a0=threadIdx.x*1e-3, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  for(int i=0;i<iters;i++){
    a0=fma(a0,s,0.5); a1=fma(a1,s,0.5); a2=fma(a2,s,0.5); a3=fma(a3,s,0.5);
    a4=fma(a4,s,0.5); a5=fma(a5,s,0.5); a6=fma(a6,s,0.5); a7=fma(a7,s,0.5);
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=a0+a1+a2+a3+a4+a5+a6+a7;
}
__global__ void fma32(float* out, int iters, float s){
  float a0=threadIdx.x*1e-3f, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  for(int i=0;i<iters;i++){
    a0=fmaf(a0,s,0.5f); a1=fmaf(a1,s,0.5f); a2=fmaf(a2,s,0.5f); a3=fmaf(a3,s,0.5f);
    a4=fmaf(a4,s,0.5f); a5=fmaf(a5,s,0.5f); a6=fmaf(a6,s,0.5f); a7=fmaf(a7,s,0.5f);
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=a0+a1+a2+a3+a4+a5+a6+a7;
}
__device__ __forceinline__ uint64_t pk(float x, float y){uint64_t r; asm("mov.b64 %0,{%1,%2};":"=l"(r):"f"(x),"f"(y)); return r;}
__global__ void fma32x2(float* out, int iters, float s){
  float b=threadIdx.x*1e-3f;
  uint64_t a0=pk(b,b+1),a1=pk(b+2,b+3),a2=pk(b+4,b+5),a3=pk(b+6,b+7),a4=pk(b+8,b+9),a5=pk(b+10,b+11),a6=pk(b+12,b+13),a7=pk(b+14,b+15);
  uint64_t ss=pk(s,s), hh=pk(0.5f,0.5f);
  for(int i=0;i<iters;i++){
#define F(a) asm("fma.rn.f32x2 %0,%0,%1,%2;":"+l"(a):"l"(ss),"l"(hh));
    F(a0)F(a1)F(a2)F(a3)F(a4)F(a5)F(a6)F(a7)
  }
  uint64_t t=a0^a1^a2^a3^a4^a5^a6^a7; float x,y; asm("mov.b64 {%0,%1},%2;":"=f"(x),"=f"(y):"l"(t));
  out[blockIdx.x*blockDim.x+threadIdx.x]=x+y;
}
__global__ void sincos32(float* out, int iters){
  float a=threadIdx.x*1e-3f, acc=0;
  for(int i=0;i<iters;i++){ float s,c; __sincosf(a,&s,&c); acc+=s*c; a+=0.37f; }
  out[blockIdx.x*blockDim.x+threadIdx.x]=acc;
}
__global__ void barrier_k(unsigned* count, volatile unsigned* gen, int nb, unsigned long long* err, unsigned long long timeout_ns){
  for(int it=0; it<nb; ++it){
    __syncthreads();
    if(threadIdx.x==0){
      unsigned g = *gen;
      __threadfence();
      unsigned a = atomicAdd(count,1u);
      if(a==gridDim.x-1){ *count=0; __threadfence(); atomicAdd((unsigned*)gen,1u); }
      else {
        unsigned long long t0; asm volatile("mov.u64 %0, %%globaltimer;":"=l"(t0));
        while(*gen==g){ unsigned long long t; asm volatile("mov.u64 %0, %%globaltimer;":"=l"(t)); if(t-t0>timeout_ns){ atomicAdd(err,1ull); return; } }
      }
      __threadfence();
    }
    __syncthreads();
  }
}
// Latency of dependent FP64 operations in one thread (clock64 cycles per operation).
__global__ void lat64(double* out, long long* cyc, int n, double x0){
  double x = x0, y = 1.000001;
  long long t0 = clock64();
  for(int i=0;i<n;i++) x = fma(x, y, 1e-9);
  long long t1 = clock64();
  for(int i=0;i<n;i++) x = 1.0 / (x + 1.5);
  long long t2 = clock64();
  for(int i=0;i<n;i++) x = sqrt(x + 2.0);
  long long t3 = clock64();
  for(int i=0;i<n;i++) x = pow(x + 1.1, -0.2);
  long long t4 = clock64();
  float f = (float)x;
  for(int i=0;i<n;i++) f = fmaf(f, 1.000001f, 1e-9f);
  long long t5 = clock64();
  out[0] = x + f; cyc[0] = t1-t0; cyc[1] = t2-t1; cyc[2] = t3-t2; cyc[3] = t4-t3; cyc[4] = t5-t4;
}
int main(){
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0));
  printf("name %s SMs %d L2 %d MB smemPerBlockOptin %zu regsPerSM %d\n", p.name, p.multiProcessorCount, p.l2CacheSize>>20, p.sharedMemPerBlockOptin, p.regsPerMultiprocessor);
  int nsm=p.multiProcessorCount;
  float* o; CK(cudaMalloc(&o, 1<<26));
  cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b); float ms;
  int blocks=nsm*4, th=512, it=4096;
  for(int rep=0;rep<2;rep++){
  fma64<<<blocks,th>>>((double*)o,it,0.999); CK(cudaDeviceSynchronize());
  cudaEventRecord(a); fma64<<<blocks,th>>>((double*)o,it,0.999); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
  printf("fp64 fma: %.3f TFLOP/s (%.3f ms)\n", 2.0*8*it*(double)blocks*th/ms/1e9, ms);
  cudaEventRecord(a); fma32<<<blocks,th>>>(o,it*8,0.999f); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
  printf("fp32 fma: %.3f TFLOP/s\n", 2.0*8*it*8*(double)blocks*th/ms/1e9);
  cudaEventRecord(a); fma32x2<<<blocks,th>>>(o,it*8,0.999f); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
  printf("fp32x2 fma: %.3f TFLOP/s\n", 2.0*16*it*8*(double)blocks*th/ms/1e9);
  cudaEventRecord(a); sincos32<<<blocks,th>>>(o,it*4); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
  printf("__sincosf: %.3f Tpairs/s\n", (double)it*4*blocks*th/ms/1e9);
  }
  unsigned* cnt; CK(cudaMalloc(&cnt, 256)); CK(cudaMemset(cnt,0,256));
  unsigned long long* err; CK(cudaMalloc(&err, 8)); CK(cudaMemset(err,0,8));
  for(int bps=1; bps<=4; bps*=2){
    int G=nsm*bps, nb=2000; void* args[]={&cnt,(void*)0,&nb,&err,0};
    unsigned* gen=cnt+16; unsigned long long to=200000000ull; args[1]=&gen; args[4]=&to;
    CK(cudaLaunchCooperativeKernel((void*)barrier_k, G, 256, args, 0, 0)); CK(cudaDeviceSynchronize());
    cudaEventRecord(a); CK(cudaLaunchCooperativeKernel((void*)barrier_k, G, 256, args, 0, 0)); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
    unsigned long long he; cudaMemcpy(&he,err,8,cudaMemcpyDeviceToHost);
    printf("grid barrier G=%d: %.3f us/barrier (timeouts %llu)\n", G, ms*1e3/nb, he);
  }
  {
    double* od; long long* cy; CK(cudaMalloc(&od, 64)); CK(cudaMalloc(&cy, 64));
    for (int rep = 0; rep < 2; ++rep) {
      lat64<<<1,1>>>(od, cy, 256, 0.5); CK(cudaDeviceSynchronize());
      long long hc[5]; cudaMemcpy(hc, cy, sizeof(hc), cudaMemcpyDeviceToHost);
      if (rep) printf("dependent-op latency (cycles/op): dfma %.1f ddiv %.1f dsqrt %.1f pow %.1f ffma %.1f\n",
                      hc[0]/256.0, hc[1]/256.0, hc[2]/256.0, hc[3]/256.0, hc[4]/256.0);
    }
  }
  size_t N=1ull<<28; float *x,*y; CK(cudaMalloc(&x,N*4)); CK(cudaMalloc(&y,N*4)); CK(cudaMemset(x,0,N*4));
  for(int r=0;r<3;r++){ cudaEventRecord(a); cudaMemcpyAsync(y,x,N*4,cudaMemcpyDeviceToDevice); cudaEventRecord(b); CK(cudaEventSynchronize(b)); cudaEventElapsedTime(&ms,a,b);
  printf("d2d copy %.1f GB/s\n", 2.0*N*4/ms/1e6); }
  return 0;
}
