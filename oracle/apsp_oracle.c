/*
 * CPU oracle for warm-start APSP: textbook Floyd-Warshall and dense
 * array-based Dijkstra, in int64 (for integer weights) and fp64 (for float
 * weights).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * The paper compares every warm-start result against a cold recomputation of
 * the APSP matrix of the updated graph by Floyd-Warshall (Section 3.2,
 * Algorithm 5, and the ratio of Eq. (equ:ratioo) in Section 5); Dijkstra's
 * algorithm is the per-source solver that Algorithm 5 runs on G - G_k.  Both are
 * written here in their plain textbook form: no blocking, no reordering.
 *
 * Conventions: matrices are dense row-major n x n.  A missing edge is
 * ORACLE_INF_I64 (int64) or +infinity (fp64).  The diagonal of a live node is
 * 0; a dead slot has an all-missing row and column (its diagonal is missing
 * too), so it takes part in no path.
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_INF_I64 ((int64_t)1 << 60)

/* Floyd-Warshall, in place: for every k, for every i, j:
 * D[i][j] = min(D[i][j], D[i][k] + D[k][j]).  Integer sums are exact. */
void oracle_fw_i64(int64_t n, int64_t *D)
{
    for (int64_t k = 0; k < n; ++k) {
        const int64_t *Dk = D + k * n;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            int64_t *Di = D + i * n;
            int64_t dik = Di[k];
            if (dik >= ORACLE_INF_I64) continue;
            for (int64_t j = 0; j < n; ++j) {
                int64_t dkj = Dk[j];
                if (dkj >= ORACLE_INF_I64) continue;
                int64_t s = dik + dkj;
                if (s < Di[j]) Di[j] = s;
            }
        }
    }
}

void oracle_fw_f64(int64_t n, double *D)
{
    for (int64_t k = 0; k < n; ++k) {
        const double *Dk = D + k * n;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double *Di = D + i * n;
            double dik = Di[k];
            if (isinf(dik)) continue;
            for (int64_t j = 0; j < n; ++j) {
                double s = dik + Dk[j];
                if (s < Di[j]) Di[j] = s;
            }
        }
    }
}

/* Dijkstra from one source on a dense adjacency matrix, O(n^2), no heap:
 * repeatedly settle the unsettled node of least tentative distance and relax
 * every edge leaving it. */
static void dijkstra_one_i64(int64_t n, const int64_t *W, int64_t s, int64_t *dist, unsigned char *done)
{
    for (int64_t v = 0; v < n; ++v) { dist[v] = ORACLE_INF_I64; done[v] = 0; }
    if (W[s * n + s] >= ORACLE_INF_I64) return;  /* dead source: reaches nothing */
    dist[s] = 0;
    for (int64_t it = 0; it < n; ++it) {
        int64_t u = -1, best = ORACLE_INF_I64;
        for (int64_t v = 0; v < n; ++v)
            if (!done[v] && dist[v] < best) { best = dist[v]; u = v; }
        if (u < 0) break;
        done[u] = 1;
        const int64_t *Wu = W + u * n;
        for (int64_t v = 0; v < n; ++v) {
            if (done[v] || Wu[v] >= ORACLE_INF_I64) continue;
            int64_t c = best + Wu[v];
            if (c < dist[v]) dist[v] = c;
        }
    }
}

static void dijkstra_one_f64(int64_t n, const double *W, int64_t s, double *dist, unsigned char *done)
{
    for (int64_t v = 0; v < n; ++v) { dist[v] = INFINITY; done[v] = 0; }
    if (isinf(W[s * n + s])) return;
    dist[s] = 0.0;
    for (int64_t it = 0; it < n; ++it) {
        int64_t u = -1;
        double best = INFINITY;
        for (int64_t v = 0; v < n; ++v)
            if (!done[v] && dist[v] < best) { best = dist[v]; u = v; }
        if (u < 0) break;
        done[u] = 1;
        const double *Wu = W + u * n;
        for (int64_t v = 0; v < n; ++v) {
            if (done[v]) continue;
            double c = best + Wu[v];
            if (c < dist[v]) dist[v] = c;
        }
    }
}

/* Rows `src[0..ns)` of the APSP matrix, one Dijkstra per source. */
void oracle_dijkstra_rows_i64(int64_t n, const int64_t *W, int64_t ns, const int64_t *src, int64_t *out)
{
#pragma omp parallel
    {
        unsigned char *done = (unsigned char *)malloc((size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < ns; ++r)
            dijkstra_one_i64(n, W, src[r], out + r * n, done);
        free(done);
    }
}

void oracle_dijkstra_rows_f64(int64_t n, const double *W, int64_t ns, const int64_t *src, double *out)
{
#pragma omp parallel
    {
        unsigned char *done = (unsigned char *)malloc((size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < ns; ++r)
            dijkstra_one_f64(n, W, src[r], out + r * n, done);
        free(done);
    }
}

int oracle_num_threads(void)
{
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            t = omp_get_num_threads();
#endif
        }
    }
    return t;
}
