// Throughput microbenchmark of the arithmetic pipes the lattice Green's function
// kernels can use on this GPU: FP64 DFMA, FP32 FFMA and its packed two-wide form
// (fma.rn.f32x2), the FP64 tensor path (mma.sync .f64 in the shapes m8n8k4,
// m16n8k4, m16n8k8 and m16n8k16) and TF32 mma.sync m16n8k8.  Every thread runs
// independent FMA / MMA chains in a loop; the rate is counted flops / CUDA-event
// time.  Run by `python bench.py --peaks`.
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1;}}while(0)

template<int CH>
__global__ void k_dfma(double* out, int iters, double a, double b){
  double x[CH];
  #pragma unroll
  for(int c=0;c<CH;c++) x[c]=threadIdx.x*1e-3+c;
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++) x[c]=fma(x[c],a,b);
  }
  double s=0;
  #pragma unroll
  for(int c=0;c<CH;c++) s+=x[c];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
template<int CH>
__global__ void k_ffma(float* out, int iters, float a, float b){
  float x[CH];
  #pragma unroll
  for(int c=0;c<CH;c++) x[c]=threadIdx.x*1e-3f+c;
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++) x[c]=fmaf(x[c],a,b);
  }
  float s=0;
  #pragma unroll
  for(int c=0;c<CH;c++) s+=x[c];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// Packed FP32: fma.rn.f32x2 on 64-bit register pairs, two FMAs per instruction.
template<int CH>
__global__ void k_ffma2(float* out, int iters, float a, float b){
  unsigned long long x[CH], av, bv;
  asm("mov.b64 %0, {%1, %2};" : "=l"(av) : "f"(a), "f"(a));
  asm("mov.b64 %0, {%1, %2};" : "=l"(bv) : "f"(b), "f"(b));
  #pragma unroll
  for(int c=0;c<CH;c++){ float v=threadIdx.x*1e-3f+c; asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(v), "f"(v+0.5f)); }
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
  }
  float s=0;
  #pragma unroll
  for(int c=0;c<CH;c++){ float lo, hi; asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c])); s+=lo+hi; }
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// DMMA m16n8k4: A 16x4 (2 f64/thread), B 4x8 (1), C/D 16x8 (4)
template<int CH>
__global__ void k_dmma16k4(double* out, int iters){
  double a0=threadIdx.x*1e-3, a1=a0+0.5, b=1.0-threadIdx.x*1e-4;
  double c[CH][4];
  #pragma unroll
  for(int q=0;q<CH;q++){c[q][0]=c[q][1]=c[q][2]=c[q][3]=0;}
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int q=0;q<CH;q++)
      asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+d"(c[q][0]), "+d"(c[q][1]), "+d"(c[q][2]), "+d"(c[q][3]) : "d"(a0), "d"(a1), "d"(b));
  }
  double s=0;
  #pragma unroll
  for(int q=0;q<CH;q++) s+=c[q][0]+c[q][1]+c[q][2]+c[q][3];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// DMMA m16n8k8: A 16x8 (4 f64/thread), B 8x8 (2), C/D 16x8 (4)
template<int CH>
__global__ void k_dmma16k8(double* out, int iters){
  double a0=threadIdx.x*1e-3, a1=a0+0.5, a2=a0+0.25, a3=a0+0.125, b0=1.0-threadIdx.x*1e-4, b1=b0*0.5;
  double c[CH][4];
  #pragma unroll
  for(int q=0;q<CH;q++){c[q][0]=c[q][1]=c[q][2]=c[q][3]=0;}
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int q=0;q<CH;q++)
      asm volatile("mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+d"(c[q][0]), "+d"(c[q][1]), "+d"(c[q][2]), "+d"(c[q][3]) : "d"(a0), "d"(a1), "d"(a2), "d"(a3), "d"(b0), "d"(b1));
  }
  double s=0;
  #pragma unroll
  for(int q=0;q<CH;q++) s+=c[q][0]+c[q][1]+c[q][2]+c[q][3];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// DMMA m16n8k16: A 16x16 (8 f64/thread), B 16x8 (4), C/D 16x8 (4)
template<int CH>
__global__ void k_dmma16k16(double* out, int iters){
  double a[8], b[4];
  #pragma unroll
  for(int t=0;t<8;t++) a[t]=threadIdx.x*1e-3+t*0.125;
  #pragma unroll
  for(int t=0;t<4;t++) b[t]=1.0-threadIdx.x*1e-4-t*0.0625;
  double c[CH][4];
  #pragma unroll
  for(int q=0;q<CH;q++){c[q][0]=c[q][1]=c[q][2]=c[q][3]=0;}
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int q=0;q<CH;q++)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
        : "+d"(c[q][0]), "+d"(c[q][1]), "+d"(c[q][2]), "+d"(c[q][3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
          "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
  }
  double s=0;
  #pragma unroll
  for(int q=0;q<CH;q++) s+=c[q][0]+c[q][1]+c[q][2]+c[q][3];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// DMMA m8n8k4: A 8x4 (1 f64/thread), B 4x8 (1 f64/thread), C/D 8x8 (2 f64/thread)
template<int CH>
__global__ void k_dmma(double* out, int iters){
  double a=threadIdx.x*1e-3, b=1.0-threadIdx.x*1e-4;
  double c0[CH], c1[CH];
  #pragma unroll
  for(int c=0;c<CH;c++){c0[c]=0;c1[c]=0;}
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++){
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
        : "+d"(c0[c]), "+d"(c1[c]) : "d"(a), "d"(b));
    }
  }
  double s=0;
  #pragma unroll
  for(int c=0;c<CH;c++) s+=c0[c]+c1[c];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// TF32 m16n8k8: A 4 regs, B 2 regs, C 4 f32
template<int CH>
__global__ void k_tf32(float* out, int iters){
  unsigned a0=0x3f800000u+threadIdx.x, a1=a0, a2=a0, a3=a0, b0=0x3f000000u, b1=b0;
  float c[CH][4];
  #pragma unroll
  for(int q=0;q<CH;q++){c[q][0]=c[q][1]=c[q][2]=c[q][3]=0.f;}
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int q=0;q<CH;q++){
      asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[q][0]), "+f"(c[q][1]), "+f"(c[q][2]), "+f"(c[q][3]) : "r"(a0),"r"(a1),"r"(a2),"r"(a3),"r"(b0),"r"(b1));
    }
  }
  float s=0;
  #pragma unroll
  for(int q=0;q<CH;q++) s+=c[q][0]+c[q][1]+c[q][2]+c[q][3];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}

int main(){
  int dev=0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,dev));
  int sms=p.multiProcessorCount;
  printf("device %s sms %d cc %d.%d\n", p.name, sms, p.major, p.minor);
  double* dout; CK(cudaMalloc(&dout, sizeof(double)*sms*64*1024));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  const int TH=256;
  for(int bps : {1,2,4,8}){
    int blocks=sms*bps; int iters=2000;
    k_dfma<8><<<blocks,TH>>>(dout,10,1.0000001,1e-9); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_dfma<8><<<blocks,TH>>>(dout,iters,1.0000001,1e-9); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl=2.0*8*iters*(double)blocks*TH;
    printf("DFMA blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bps, ms, fl/ms/1e9);
  }
  for(int bps : {2,4,8}){
    int blocks=sms*bps; int iters=20000;
    k_ffma<8><<<blocks,TH>>>((float*)dout,10,1.0000001f,1e-9f); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_ffma<8><<<blocks,TH>>>((float*)dout,iters,1.0000001f,1e-9f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl=2.0*8*iters*(double)blocks*TH;
    printf("FFMA blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bps, ms, fl/ms/1e9);
  }
  for(int bps : {2,4,8}){
    int blocks=sms*bps; int iters=20000;
    k_ffma2<8><<<blocks,TH>>>((float*)dout,10,1.0000001f,1e-9f); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_ffma2<8><<<blocks,TH>>>((float*)dout,iters,1.0000001f,1e-9f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl=2.0*2*8*iters*(double)blocks*TH;
    printf("FFMA2 (fma.rn.f32x2) blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bps, ms, fl/ms/1e9);
  }
  for(int bps : {1,2,4}){
    int blocks=sms*bps; int iters=200;
    k_dmma16k4<4><<<blocks,TH>>>(dout,10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_dmma16k4<4><<<blocks,TH>>>(dout,iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl=2.0*16*8*4*4.0*iters*(double)blocks*(TH/32);
    printf("DMMA m16n8k4 blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bps, ms, fl/ms/1e9);
    k_dmma16k8<4><<<blocks,TH>>>(dout,10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_dmma16k8<4><<<blocks,TH>>>(dout,iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    fl=2.0*16*8*8*4.0*iters*(double)blocks*(TH/32);
    printf("DMMA m16n8k8 blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bps, ms, fl/ms/1e9);
    k_dmma16k16<4><<<blocks,TH>>>(dout,10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_dmma16k16<4><<<blocks,TH>>>(dout,iters/2); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    fl=2.0*16*8*16*4.0*(iters/2)*(double)blocks*(TH/32);
    printf("DMMA m16n8k16 blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bps, ms, fl/ms/1e9);
  }
  for(int bps : {1,2,4,8}){
    int blocks=sms*bps; int iters=500;
    k_dmma<4><<<blocks,TH>>>(dout,10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_dmma<4><<<blocks,TH>>>(dout,iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl=2.0*8*8*4*4.0*iters*(double)blocks*(TH/32);
    printf("DMMA m8n8k4 blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bps, ms, fl/ms/1e9);
  }
  for(int bps : {2,4,8}){
    int blocks=sms*bps; int iters=20000;
    k_tf32<4><<<blocks,TH>>>((float*)dout,10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); k_tf32<4><<<blocks,TH>>>((float*)dout,iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl=2.0*16*8*8*4.0*iters*(double)blocks*(TH/32);
    printf("TF32 mma.sync m16n8k8 blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bps, ms, fl/ms/1e9);
  }
  CK(cudaGetLastError());
  return 0;
}
