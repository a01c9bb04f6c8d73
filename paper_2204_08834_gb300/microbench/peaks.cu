// peaks.cu - throughput micro-benchmark: FP64 DFMA/DADD, FP32 FFMA, FP64<->FP32 conversion, FP64
// division, HBM copy, and 256-byte strided tile copies (the access pattern of the y/z passes).
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o peaks peaks.cu
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s at %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

template<int OP>
__global__ void alu(double* out, int iters, double s) {
  double a0 = threadIdx.x*1e-3, a1=a0+1, a2=a0+2, a3=a0+3, a4=a0+4, a5=a0+5, a6=a0+6, a7=a0+7;
  float f0=a0,f1=a1,f2=a2,f3=a3,f4=a4,f5=a5,f6=a6,f7=a7;
  for (int it=0; it<iters; ++it) {
    if (OP==0) { // DFMA
      a0=fma(a0,s,1.0); a1=fma(a1,s,1.0); a2=fma(a2,s,1.0); a3=fma(a3,s,1.0);
      a4=fma(a4,s,1.0); a5=fma(a5,s,1.0); a6=fma(a6,s,1.0); a7=fma(a7,s,1.0);
    } else if (OP==1) { // DADD
      a0+=s; a1+=s; a2+=s; a3+=s; a4+=s; a5+=s; a6+=s; a7+=s;
    } else if (OP==2) { // FFMA
      float fs=(float)s;
      f0=fmaf(f0,fs,1.f); f1=fmaf(f1,fs,1.f); f2=fmaf(f2,fs,1.f); f3=fmaf(f3,fs,1.f);
      f4=fmaf(f4,fs,1.f); f5=fmaf(f5,fs,1.f); f6=fmaf(f6,fs,1.f); f7=fmaf(f7,fs,1.f);
    } else if (OP==3) { // F2F f64->f32->f64 (2 conversions each)
      a0=(double)(float)a0+s; a1=(double)(float)a1+s; a2=(double)(float)a2+s; a3=(double)(float)a3+s;
    } else if (OP==4) { // DDIV
      a0=s/a0; a1=s/a1; a2=s/a2; a3=s/a3;
    }
  }
  double r = a0+a1+a2+a3+a4+a5+a6+a7 + f0+f1+f2+f3+f4+f5+f6+f7;
  if (r == 123.456) out[threadIdx.x] = r;
}

__global__ void copyk(const float4* __restrict__ a, float4* __restrict__ b, size_t n) {
  size_t i = blockIdx.x*(size_t)blockDim.x + threadIdx.x, st = (size_t)gridDim.x*blockDim.x;
  for (; i<n; i+=st) b[i]=a[i];
}
// read rows of 'w' float2 (chunk) from each of R rows with stride 'stride' float2; tiles over columns and planes
__global__ void strided(const float2* __restrict__ a, float2* __restrict__ b, int nrows, int ncol, int nplanes) {
  // block: tile of 32 columns x nrows, one plane; thread reads column c, rows r..
  int tiles = ncol/32;
  int tile = blockIdx.x % tiles, plane = blockIdx.x / tiles;
  const float2* src = a + (size_t)plane*nrows*ncol + tile*32;
  float2* dst = b + (size_t)plane*nrows*ncol + tile*32;
  for (int r = threadIdx.y; r < nrows; r += blockDim.y) dst[(size_t)r*ncol + threadIdx.x] = src[(size_t)r*ncol + threadIdx.x];
}

int main() {
  int dev=0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,dev));
  printf("%s SMs=%d clock? l2=%d MB smem/blk optin=%zu\n", p.name, p.multiProcessorCount, p.l2CacheSize>>20, p.sharedMemPerBlockOptin);
  double* out; CK(cudaMalloc(&out, 4096*8));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  int blocks = p.multiProcessorCount*8, threads=256, iters=4096; float ms;
  const char* names[5]={"DFMA","DADD","FFMA","F2F(x2)","DDIV"};
  int opsPer[5]={8,8,8,8,4};
  for (int op=0; op<5; ++op) {
    for (int rep=0; rep<2; ++rep) {
      cudaEventRecord(e0);
      switch(op){case 0: alu<0><<<blocks,threads>>>(out,iters,0.999); break; case 1: alu<1><<<blocks,threads>>>(out,iters,0.999); break;
        case 2: alu<2><<<blocks,threads>>>(out,iters,0.999); break; case 3: alu<3><<<blocks,threads>>>(out,iters/4,0.999); break;
        case 4: alu<4><<<blocks,threads>>>(out,iters/16,0.999); break;}
      cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    }
    double it = (op==3)? iters/4 : (op==4? iters/16: iters);
    double lanes = (double)blocks*threads*it*opsPer[op];
    printf("%-8s %.3f Glane-op/s  (%.2f ms)\n", names[op], lanes/ms/1e6, ms);
  }
  size_t nbytes = (size_t)4<<30; float4 *a,*b; CK(cudaMalloc(&a,nbytes)); CK(cudaMalloc(&b,nbytes));
  cudaMemset(a,0,nbytes); cudaMemset(b,0,nbytes);
  for (int rep=0; rep<3; ++rep) { cudaEventRecord(e0); copyk<<<p.multiProcessorCount*16,512>>>(a,b,nbytes/16); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);}
  printf("copy %.1f GB/s\n", 2.0*nbytes/ms/1e6);
  // strided: planes of 512 rows x 256 float2 columns  (2 KB row stride) -> 4 GiB / (512*256*8) planes
  int nrows=512, ncol=256; int nplanes = (int)(nbytes/((size_t)nrows*ncol*8));
  for (int rep=0; rep<3; ++rep) { cudaEventRecord(e0); strided<<<nplanes*(ncol/32), dim3(32,16)>>>((float2*)a,(float2*)b,nrows,ncol,nplanes); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);}
  printf("strided-256B-tiles copy %.1f GB/s\n", 2.0*nbytes/ms/1e6);
  // z-like: stride = 512 rows * 257 ... use ncol=256*512 (rows are planes)
  { int nr=512, nc=256*64; int np=(int)(nbytes/((size_t)nr*nc*8));
    for (int rep=0; rep<3; ++rep) { cudaEventRecord(e0); strided<<<np*(nc/32), dim3(32,16)>>>((float2*)a,(float2*)b,nr,nc,np); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);}
    printf("strided-256B-tiles (large stride %d KB) copy %.1f GB/s\n", nc*8/1024, 2.0*nbytes/ms/1e6); }
  CK(cudaGetLastError());
  printf("done\n");
  return 0;
}
