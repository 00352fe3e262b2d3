// Random-row gather ceiling of this GPU: the bandwidth of reading 64-byte rows
// at random indices from an 8.6 GB array, the access pattern of the union
// pass.  Three index laws: uniform; the in-degree law of an R-MAT graph with
// scrambled ids (hot rows scattered); the same law with ids ranked by
// popularity (hot rows packed, as hanf_create stores counters).  U = rows in
// flight per 4-lane group.  Reference for the union kernel's roofline beside
// the copy bandwidth.  Built and run by bench.py --gather-ceiling.
#include <cstdio>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s %s\n",#x,cudaGetErrorString(e)); return 1;}}while(0)

__device__ __forceinline__ uint32_t bmax(uint32_t a, uint32_t b){
  uint32_t d=(a|0x80808080u)-b, m; asm("prmt.b32 %0, %1, %2, %3;":"=r"(m):"r"(d),"r"(0u),"r"(0xBA98u)); return (a&m)|(b&~m);}

// U rows in flight per lane group (4 lanes x 16 B = one row)
template<int U>
__global__ void gather(const uint4* __restrict__ rows, const uint32_t* __restrict__ idx, int64_t m, uint4* out){
  int lane=threadIdx.x&31, g=lane>>2, gl=lane&3;
  int64_t warp=(blockIdx.x*(int64_t)blockDim.x+threadIdx.x)>>5, nw=((int64_t)gridDim.x*blockDim.x)>>5;
  uint4 acc=make_uint4(0,0,0,0);
  // each warp handles chunks of 8*U indices; group g takes indices g, g+8, ...
  for(int64_t base=warp*8*U; base<m; base+=nw*8*U){
    uint32_t w[U];
    #pragma unroll
    for(int u=0;u<U;++u){ int64_t i=base+g+8*u; w[u]= i<m ? __ldg(idx+i) : 0xffffffffu; }
    uint4 x[U];
    #pragma unroll
    for(int u=0;u<U;++u) if(w[u]!=0xffffffffu) x[u]=__ldg(rows+(int64_t)w[u]*4+gl); else x[u]=make_uint4(0,0,0,0);
    #pragma unroll
    for(int u=0;u<U;++u){acc.x=bmax(acc.x,x[u].x);acc.y=bmax(acc.y,x[u].y);acc.z=bmax(acc.z,x[u].z);acc.w=bmax(acc.w,x[u].w);}
  }
  if(acc.x==0x12345678u) out[0]=acc;  // keeps the loads alive
}

__global__ void fill_idx(uint32_t* idx, int64_t m, uint32_t nrows, int skew){
  // skew 0: uniform; 1: R-MAT target law (each of 27 bits is 1 w.p. 0.24), ids scrambled;
  // 2: same law with ids ranked by popularity (fewest one-bits first) -- "relabelled"
  for(int64_t i=blockIdx.x*(int64_t)blockDim.x+threadIdx.x;i<m;i+=(int64_t)gridDim.x*blockDim.x){
    uint64_t z=i+0x9E3779B97F4A7C15ull; z=(z^(z>>30))*0xBF58476D1CE4E5B9ull; z=(z^(z>>27))*0x94D049BB133111EBull; z^=z>>31;
    if(skew==0){ idx[i]=(uint32_t)(((z>>11)*0x1p-53)*nrows)%nrows; continue; }
    uint32_t id=0; uint64_t s=z;
    for(int b=0;b<27;++b){ s=s*6364136223846793005ull+1442695040888963407ull; double u=(s>>11)*0x1p-53; id=(id<<1)|(u<0.24?1u:0u); }
    if(skew==1){ uint64_t y=((uint64_t)id*0x9E3779B1ull)&((1ull<<27)-1); idx[i]=(uint32_t)(y%nrows); continue; }
    // rank: ids ordered by popcount, then by value: offset of class k = sum_{j<k} C(27,j)
    int k=__popc(id); uint64_t off=0, c=1; for(int j=0;j<k;++j){ off+=c; c=c*(27-j)/(j+1); }
    // position inside the class: a hash of id mod C(27,k)
    uint64_t pos=((uint64_t)id*0x9E3779B97F4A7C15ull>>20)%c;
    idx[i]=(uint32_t)((off+pos)%nrows);
  }
}
__global__ void copyk(const uint4* a, uint4* b, int64_t n){ for(int64_t i=blockIdx.x*(int64_t)blockDim.x+threadIdx.x;i<n;i+=(int64_t)gridDim.x*blockDim.x) b[i]=a[i]; }

template<int U> float run(const uint4* rows, const uint32_t* idx, int64_t m, uint4* out, int blocks){
  cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b);
  gather<U><<<blocks,256>>>(rows,idx,m,out);
  cudaEventRecord(a); for(int r=0;r<3;++r) gather<U><<<blocks,256>>>(rows,idx,m,out); cudaEventRecord(b); cudaEventSynchronize(b);
  float ms; cudaEventElapsedTime(&ms,a,b); return ms/3;
}

int main(){
  int nsm; cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  const int64_t m = 1ll<<28;             // gathers per launch
  uint32_t* idx; uint4* out; CK(cudaMalloc(&idx, m*4)); CK(cudaMalloc(&out, 64));
  for (int64_t nrows : {1ll<<27}) {
    uint4* rows; CK(cudaMalloc(&rows, nrows*64)); CK(cudaMemset(rows, 1, nrows*64));
    for (int skew=0; skew<3; ++skew) {
      fill_idx<<<nsm*16,256>>>(idx, m, (uint32_t)nrows, skew); CK(cudaDeviceSynchronize());
      for (int bpsm : {4}) {
        int blocks = nsm*bpsm;
        float t1=run<1>(rows,idx,m,out,blocks), t4=run<4>(rows,idx,m,out,blocks), t8=run<8>(rows,idx,m,out,blocks), t16=run<16>(rows,idx,m,out,blocks);
        double gb = m*64.0/1e9;
        printf("rows=%lld (%.1f GB) skew=%d blocks/SM=%d  GB/s row bytes: U1 %.0f  U4 %.0f  U8 %.0f  U16 %.0f\n",
               (long long)nrows, nrows*64/1e9, skew, bpsm, gb/(t1/1e3), gb/(t4/1e3), gb/(t8/1e3), gb/(t16/1e3));
      }
    }
    CK(cudaGetLastError());
    CK(cudaFree(rows));
  }
  { int64_t n=1ll<<30; uint4 *a,*b; CK(cudaMalloc(&a,n)); CK(cudaMalloc(&b,n)); cudaMemset(a,0,n);
    cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    copyk<<<nsm*8,256>>>(a,b,n/16); cudaEventRecord(e0); for(int r=0;r<5;++r) copyk<<<nsm*8,256>>>(a,b,n/16); cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms,e0,e1); printf("copy 1 GiB: %.0f GB/s (read+write)\n", 2.0*n*5/(ms/1e3)/1e9); }
  CK(cudaDeviceSynchronize());
  return 0;
}
