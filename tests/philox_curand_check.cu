// Test helper: prints curand's host-callable Philox4x32-10 for counters/keys read
// from stdin, to check the oracle's own Philox against the CUDA library routine.
#define QUALIFIERS static __forceinline__ __host__ __device__
#include <curand_philox4x32_x.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char** argv) {
  // reads lines "c0 c1 c2 c3 k0 k1" (hex) from stdin, prints the Philox output
  unsigned a[6];
  while (scanf("%x %x %x %x %x %x", &a[0],&a[1],&a[2],&a[3],&a[4],&a[5]) == 6) {
    uint4 c = make_uint4(a[0],a[1],a[2],a[3]); uint2 k = make_uint2(a[4],a[5]);
    uint4 o = curand_Philox4x32_10(c, k);
    printf("%08x %08x %08x %08x\n", o.x, o.y, o.z, o.w);
  }
  return 0;
}
