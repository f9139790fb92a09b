"""The oracle's C part under AddressSanitizer and UndefinedBehaviorSanitizer:
a small C driver runs Floyd-Warshall and the Dijkstra rows (int64 and fp64,
with missing edges and dead slots) and checks them against Bellman-Ford
written in the driver; any out-of-bounds access, overflow or other undefined
behaviour aborts the run."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "apsp_oracle.c")

DRIVER = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <math.h>
#define INF ((int64_t)1 << 60)
void oracle_fw_i64(int64_t n, int64_t *D);
void oracle_fw_f64(int64_t n, double *D);
void oracle_dijkstra_rows_i64(int64_t n, const int64_t *W, int64_t ns, const int64_t *src, int64_t *out);
void oracle_dijkstra_rows_f64(int64_t n, const double *W, int64_t ns, const int64_t *src, double *out);

static uint64_t state = 88172645463325252ull;
static uint64_t next(void) { state ^= state << 13; state ^= state >> 7; state ^= state << 17; return state; }

/* Bellman-Ford from s over the dense matrix (missing = INF / inf). */
static void bf_i64(int n, const int64_t *W, int s, int64_t *d) {
    for (int v = 0; v < n; ++v) d[v] = INF;
    if (W[s * n + s] != 0) return;  /* dead source */
    d[s] = 0;
    for (int it = 0; it < n; ++it)
        for (int u = 0; u < n; ++u)
            if (d[u] < INF)
                for (int v = 0; v < n; ++v)
                    if (W[u * n + v] < INF && d[u] + W[u * n + v] < d[v]) d[v] = d[u] + W[u * n + v];
}
static void bf_f64(int n, const double *W, int s, double *d) {
    for (int v = 0; v < n; ++v) d[v] = INFINITY;
    if (W[s * n + s] != 0.0) return;
    d[s] = 0.0;
    for (int it = 0; it < n; ++it)
        for (int u = 0; u < n; ++u)
            if (d[u] < INFINITY)
                for (int v = 0; v < n; ++v)
                    if (d[u] + W[u * n + v] < d[v]) d[v] = d[u] + W[u * n + v];
}

int main(void) {
    for (int trial = 0; trial < 40; ++trial) {
        int n = 1 + (int)(next() % 23);
        int64_t *W = malloc(sizeof(int64_t) * n * n), *D = malloc(sizeof(int64_t) * n * n);
        double *Wf = malloc(sizeof(double) * n * n), *Df = malloc(sizeof(double) * n * n);
        int64_t *rows = malloc(sizeof(int64_t) * n * n), *src = malloc(sizeof(int64_t) * n), *ref = malloc(sizeof(int64_t) * n);
        double *rowsf = malloc(sizeof(double) * n * n), *reff = malloc(sizeof(double) * n);
        char *dead = calloc(n, 1);
        for (int v = 0; v < n; ++v) dead[v] = (next() % 7) == 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                int miss = (next() % 4) == 0 || dead[i] || dead[j];
                int64_t w = (int64_t)(next() % 10);
                W[i * n + j] = (i == j) ? (dead[i] ? INF : 0) : (miss ? INF : w);
                Wf[i * n + j] = W[i * n + j] >= INF ? INFINITY : (double)W[i * n + j] + 0.25;
                if (i == j && !dead[i]) Wf[i * n + j] = 0.0;
            }
        for (int k = 0; k < n * n; ++k) { D[k] = W[k]; Df[k] = Wf[k]; }
        oracle_fw_i64(n, D);
        oracle_fw_f64(n, Df);
        for (int s = 0; s < n; ++s) src[s] = s;
        oracle_dijkstra_rows_i64(n, W, n, src, rows);
        oracle_dijkstra_rows_f64(n, Wf, n, src, rowsf);
        for (int s = 0; s < n; ++s) {
            bf_i64(n, W, s, ref);
            bf_f64(n, Wf, s, reff);
            for (int v = 0; v < n; ++v) {
                if (D[s * n + v] != ref[v] || rows[s * n + v] != ref[v]) { printf("int mismatch %d %d\n", s, v); return 1; }
                double a = Df[s * n + v], b = rowsf[s * n + v], c = reff[v];
                if (isinf(c) ? !(isinf(a) && isinf(b)) : (fabs(a - c) > 1e-9 || fabs(b - c) > 1e-9)) {
                    printf("float mismatch %d %d\n", s, v); return 1;
                }
            }
        }
        free(W); free(D); free(Wf); free(Df); free(rows); free(src); free(ref); free(rowsf); free(reff); free(dead);
    }
    printf("ok\n");
    return 0;
}
"""


def test_oracle_c_under_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    drv = tmp_path / "driver.c"
    drv.write_text(DRIVER)
    exe = tmp_path / "oracle_sanitized"
    cmd = [gcc, "-std=c11", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=all", SRC, str(drv), "-o", str(exe), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("this gcc has no sanitizer runtime: " + r.stderr.strip().splitlines()[-1])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="halt_on_error=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert run.stdout.strip().endswith("ok")
