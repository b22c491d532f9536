"""Host-side logic shared by the CUDA solves, compiled for the host (nvcc,
no GPU needed) from the library's own header and checked against the
mathematics it restates:

- sor_omega_update: Young's relation for consistently ordered matrices
  (red-black ordering is one), checked on an explicit red-black ordered
  Laplacian-type M-matrix: the SOR spectral radius at omega < omega_b,
  computed from the iteration matrix, must give back the optimal relaxation,
  which a scan over omega finds independently;
- check_decision: the two-part stopping test (2-norm and max |r|) and the
  stop at the FP32 floor of max |r|;
- next_check_batch: the predicted spacing of the checks."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2111_11866_gb300", "csrc")

DRIVER = r'''
#include <cstdio>
#include "seg4d_internal.cuh"
using namespace seg4d_impl;
int main() {
    char op[32];
    while (std::scanf("%31s", op) == 1) {
        if (op[0] == 'w') {                       // w omega lam
            double om, lam;
            std::scanf("%lf %lf", &om, &lam);
            std::printf("%.15g\n", sor_omega_update(om, lam));
        } else if (op[0] == 'n') {                // n rn prev it prev_it tol bn ce mixed
            double rn, pr, tol, bn; int it, pit, ce, mx;
            std::scanf("%lf %lf %d %d %lf %lf %d %d", &rn, &pr, &it, &pit, &tol, &bn, &ce, &mx);
            std::printf("%d\n", next_check_batch(rn, pr, it, pit, tol, bn, ce, mx != 0));
        } else {                                  // c k, then k checks: rn bn rinf bmax it
            int k; double tol, tinf; int ce;
            std::scanf("%d %lf %lf %d", &k, &tol, &tinf, &ce);
            CheckState cs;
            for (int q = 0; q < k; ++q) {
                double rn, bn, ri, bm; int it, batch = -1;
                std::scanf("%lf %lf %lf %lf %d", &rn, &bn, &ri, &bm, &it);
                const int d = check_decision(cs, rn, bn, ri, bm, it, tol, tinf, ce, false, batch);
                std::printf("%d %d\n", d, batch);
            }
        }
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("hostlogic")
    src = d / "driver.cu"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True,
                   capture_output=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout
        return out.split("\n")

    return run


def _redblack_matrix(n=10, diag_extra=0.05):
    """Red-black ordered M-matrix of a 2D 5-point stencil (Dirichlet ends),
    diagonal 4 + diag_extra: consistently ordered."""
    idx = [(i, j) for i in range(n) for j in range(n)]
    red = [p for p in idx if (p[0] + p[1]) % 2 == 0]
    black = [p for p in idx if (p[0] + p[1]) % 2 == 1]
    order = red + black
    pos = {p: k for k, p in enumerate(order)}
    N = len(order)
    A = np.zeros((N, N))
    for (i, j), k in pos.items():
        A[k, k] = 4.0 + diag_extra
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            q = (i + di, j + dj)
            if q in pos:
                A[k, pos[q]] = -1.0
    return A, len(red)


def _sor_radius(A, omega):
    D = np.diag(np.diag(A))
    L = np.tril(A, -1)
    U = np.triu(A, 1)
    M = np.linalg.solve(D + omega * L, (1 - omega) * D - omega * U)
    return float(np.max(np.abs(np.linalg.eigvals(M))))


def test_young_relation_on_a_red_black_matrix(prog):
    A, _ = _redblack_matrix()
    J = np.eye(len(A)) - A / np.diag(A)[:, None]
    mu = float(np.max(np.abs(np.linalg.eigvals(J))))
    wb = 2.0 / (1.0 + np.sqrt(1.0 - mu * mu))
    # the optimum found by scanning the SOR radius directly
    ws = np.linspace(1.0, 1.99, 199)
    w_scan = ws[np.argmin([_sor_radius(A, w) for w in ws])]
    assert abs(w_scan - wb) < 0.01
    for om in (1.0, 1.2, 1.4):
        lam = _sor_radius(A, om)
        got = float(prog([f"w {om} {lam}"])[0])
        assert abs(got - wb) < 1e-6, (om, got, wb)


def test_omega_unchanged_past_the_optimum_and_capped(prog):
    out = prog(["w 1.8 0.8", "w 1.7 0.7", "w 1.9 0.91", "w 1.5 1.2", "w 1.5 0.0",
                "w 1.9 0.999999"])
    assert [float(x) for x in out[:5]] == [1.8, 1.7, 1.9, 1.5, 1.5]
    assert float(out[5]) == 1.95   # mu close to 1: capped


def test_two_part_stopping_test(prog):
    # checks: rn bn rinf bmax it
    out = prog(["c 3 1e-5 1e-5 10",
                "1e-3 1 1e-2 1 0",        # neither part: go on
                "5e-6 1 5e-5 1 10",       # 2-norm holds, max |r| not: go on
                "5e-6 1 5e-6 1 20"])      # both hold: stop
    dec = [tuple(int(v) for v in l.split()) for l in out[:3]]
    assert dec[0][0] == 0 and dec[1][0] == 0 and dec[2][0] == 1
    out = prog(["c 1 1e-5 0 10", "5e-6 1 0.5 1 0"])   # tol_inf = 0: the 2-norm alone
    assert int(out[0].split()[0]) == 1


def test_floor_of_max_residual_stops_the_solve(prog):
    out = prog(["c 3 1e-5 1e-6 10",
                "5e-6 1 4e-5 1 0",
                "4e-6 1 3.99e-5 1 12",    # max |r| no longer falls (>= 0.99 per sweep)
                "3e-6 1 3e-5 1 14"])
    assert int(out[1].split()[0]) == 2   # kStopFloor
    # falling fast enough: no floor stop
    out = prog(["c 2 1e-5 1e-6 10", "5e-6 1 4e-5 1 0", "4e-6 1 1e-5 1 12"])
    assert int(out[1].split()[0]) == 0


def test_check_spacing_prediction(prog):
    # contraction 0.5 per sweep over 10 sweeps; residual 1e-3 of ||b||, target
    # 1e-6: need = log(1e-3)/log(0.5) = 9.97 sweeps; plain cap 1e-3 -> 10;
    # the batch is ceil(0.8 * need) = 8
    rn, prev = 1e-3, 1e-3 * 2 ** 10
    out = prog([f"n {rn} {prev} 20 10 1e-6 1 10 0"])
    assert int(out[0]) == 8
    # no usable history: check_every
    assert int(prog(["n 1e-3 -1 0 0 1e-6 1 10 0"])[0]) == 10
