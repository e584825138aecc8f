/* A C caller of the library: no Python, only the header, the shared library
 * and the CUDA runtime.  Computes the pairs of n angles x[i] = i * 0.001 - 500
 * (binary32) with sincos_pairs and, for the same angles, exp(ix) with
 * sincos_expi; writes s, c and the interleaved z to a file as raw binary32
 * for the test to compare with the oracle.
 *
 *   c_abi_example <n> <out-file>      exit status 0 on success
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "sincos_pairs.h"

static int fail(const char *what, int rc)
{
    fprintf(stderr, "%s failed: %d (%s)\n", what, rc, rc < 0 ? sincos_strerror(rc) : "cuda");
    return 1;
}

int main(int argc, char **argv)
{
    if (argc != 3) {
        fprintf(stderr, "usage: %s n out-file\n", argv[0]);
        return 2;
    }
    const long long n = atoll(argv[1]);
    if (n <= 0) return 2;
    float *h = (float *)malloc((size_t)n * 4 * 4);
    if (!h) return 1;
    for (long long i = 0; i < n; ++i) h[i] = (float)((double)i * 0.001 - 500.0);

    float *x = NULL, *s = NULL, *c = NULL, *z = NULL;
    cudaError_t e = cudaMalloc((void **)&x, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&z, (size_t)n * 8);
    if (e == cudaSuccess) e = cudaMemcpy(x, h, (size_t)n * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail("cuda setup", (int)e);

    int rc = sincos_pairs(x, s, c, n, NULL);
    if (rc != SINCOS_OK) return fail("sincos_pairs", rc);
    rc = sincos_expi(x, z, n, SINCOS_RED_PLAIN, SINCOS_COEF_NORMALIZED, NULL);
    if (rc != SINCOS_OK) return fail("sincos_expi", rc);
    e = cudaMemcpy(h, s, (size_t)n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(h + n, c, (size_t)n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(h + 2 * n, z, (size_t)n * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail("cuda copy back", (int)e);

    FILE *f = fopen(argv[2], "wb");
    if (!f || fwrite(h, 4, (size_t)n * 4, f) != (size_t)n * 4) return fail("write", -1);
    fclose(f);
    cudaFree(x);
    cudaFree(s);
    cudaFree(c);
    cudaFree(z);
    free(h);
    printf("c_abi_example: %lld pairs, library version %d\n", n, sincos_version());
    return 0;
}
