"""Host logic of the pipelined CG's row partition and block-local
preconditioner (csrc/emu_cgpart.cu), compiled here with g++ and driven
through tests/cg_partition_harness.cpp.

The Laplacian is the scalar ACAP matrix of Eq. 4 (pinned rows identity),
assembled below from the rest geometry. Checks: the partition is a balanced
permutation into spatially split parts; the permuted system is P A P^T
without the entries that are rounding residue; the local table holds the
symmetric Jacobi-scaled diagonal blocks; the Gershgorin bound covers their
spectra; the Chebyshev coefficients reproduce the closed form
1 - lambda p(lambda) = T_k((theta - lambda) / delta) / T_k(theta / delta);
and the preconditioner is symmetric positive definite and cuts the CG
iteration count against Jacobi.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
import scipy.sparse as sp

from emu_inputs import mtu_for_tet_count
from oracle.emu_oracle import rest_geometry

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2006_08821_gb300", "csrc")
NT = 256
CHEB_MAX = 8


@pytest.fixture(scope="module")
def harness():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp(prefix="cgpart_")
    exe = os.path.join(d, "harness")
    cmd = [gxx, "-O2", "-std=c++17", "-I", CSRC, "-x", "c++", os.path.join(CSRC, "emu_cgpart.cu"), "-x", "c++",
           os.path.join(HERE, "cg_partition_harness.cpp"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    yield exe, d
    shutil.rmtree(d, ignore_errors=True)


def laplacian(mesh):
    """Scalar Laplacian L_ab = sum_i V_i gradN_a . gradN_b over free rows;
    pinned rows are identity rows (the host's layout)."""
    Q = np.asarray(mesh.rest_pos, dtype=np.float64)
    T = np.asarray(mesh.tets, dtype=np.int64)
    n = Q.shape[0]
    _, Dinv, V = rest_geometry(Q, T)
    gN = np.zeros((T.shape[0], 4, 3))
    gN[:, :3, :] = Dinv                      # rows of D_m^-1: gradients of N_0..N_2
    gN[:, 3, :] = -Dinv.sum(axis=1)
    fixed = np.zeros(n, dtype=bool)
    fixed[mesh.fixed_verts] = True
    rows, cols, vals = [], [], []
    for a in range(4):
        for b in range(4):
            lv = V * np.einsum("ij,ij->i", gN[:, a, :], gN[:, b, :])
            keep = ~fixed[T[:, a]] & ~fixed[T[:, b]]
            rows.append(T[keep, a])
            cols.append(T[keep, b])
            vals.append(lv[keep])
    fv = np.nonzero(fixed)[0]
    rows.append(fv)
    cols.append(fv)
    vals.append(np.ones(fv.size))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return Q, A


def run(harness, Q, A, G, rpt, degree):
    exe, d = harness
    n = Q.shape[0]
    fin, fout = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
    with open(fin, "wb") as f:
        np.array([n, A.nnz], dtype=np.int64).tofile(f)
        np.array([G, rpt, NT, degree], dtype=np.int32).tofile(f)
        Q.astype(np.float64).ravel().tofile(f)
        A.indptr.astype(np.int32).tofile(f)
        A.indices.astype(np.int32).tofile(f)
        A.data.astype(np.float64).tofile(f)
    subprocess.run([exe, fin, fout], check=True)
    buf = open(fout, "rb").read()
    o = 0

    def take(dtype, cnt):
        nonlocal o
        a = np.frombuffer(buf, dtype=dtype, count=cnt, offset=o)
        o += a.nbytes
        return a

    ok, G_, rpt_, nt_, lw, deg = take(np.int32, 6)
    r = dict(ok=bool(ok), G=int(G_), rpt=int(rpt_), lw=int(lw), degree=int(deg))
    r["lmax"] = float(take(np.float64, 1)[0])
    r["c0"] = float(take(np.float32, 1)[0])
    r["c1"] = take(np.float32, CHEB_MAX).astype(np.float64)
    r["c2"] = take(np.float32, CHEB_MAX).astype(np.float64)
    if not ok:
        return r
    r["perm"] = take(np.int32, n)
    r["off"] = take(np.int32, G + 1)
    nnz_p = int(take(np.int64, 1)[0])
    rp = take(np.int32, n + 1)
    cp = take(np.int32, nnz_p)
    vp = take(np.float32, nnz_p)
    r["Ap"] = sp.csr_matrix((vp, cp, rp), shape=(n, n))
    r["dinv"] = take(np.float32, n)
    nloc = int(take(np.int64, 1)[0])
    r["loc"] = take(np.uint32, nloc)
    assert o == len(buf)
    return r


def local_blocks(r):
    """Decoded local tables: per part, the dense off-diagonal block O_b."""
    G, rpt, lw = r["G"], r["rpt"], r["lw"]
    loc = r["loc"].reshape(G, rpt, lw, NT)
    out = []
    for b in range(G):
        cnt = int(r["off"][b + 1] - r["off"][b])
        O = np.zeros((cnt, cnt))
        for li in range(rpt * NT):
            k, t = divmod(li, NT)
            for e in range(lw):
                w = int(loc[b, k, e, t])
                col = w & 0xFFFF
                val = np.frombuffer(np.uint32(w & 0xFFFF0000).tobytes(), dtype=np.float32)[0]
                if li >= cnt:
                    assert val == 0.0 and col < rpt * NT  # slots past the part: weight 0
                    continue
                assert col < cnt                         # a row of the same part
                if val != 0.0:
                    O[li, col] += val
                else:
                    assert col == li or val == 0.0
        out.append(O)
    return out


def cheb_apply(r, y, O, d_inv):
    """P y = D^-1/2 x_k, x_k the Chebyshev iterate for (I + O) x = D^-1/2 y."""
    sd = np.sqrt(d_inv)
    ys = sd * y
    x = r["c0"] * ys
    dk = x.copy()
    res = ys - x - O @ x
    for i in range(1, r["degree"]):
        dk = r["c1"][i] * dk + r["c2"][i] * res
        x = x + dk
        if i + 1 < r["degree"]:
            res = res - dk - O @ dk
    return sd * x


@pytest.fixture(scope="module")
def case():
    mesh = mtu_for_tet_count(16000)
    Q, A = laplacian(mesh)
    return mesh, Q, A


def test_partition_is_a_balanced_permutation_into_compact_parts(harness, case):
    _, Q, A = case
    n = Q.shape[0]
    G = 8
    r = run(harness, Q, A, G, 2, 4)
    assert r["ok"]
    perm = r["perm"]
    np.testing.assert_array_equal(np.sort(perm), np.arange(n))
    sizes = np.diff(r["off"])
    assert sizes.sum() == n and sizes.max() - sizes.min() <= 1 and sizes.max() <= 2 * NT
    # recursive bisection: the parts' bounding boxes are small against the mesh's
    ext = Q.max(0) - Q.min(0)
    for b in range(G):
        P = Q[perm[r["off"][b]:r["off"][b + 1]]]
        assert np.prod(P.max(0) - P.min(0)) <= 0.25 * np.prod(ext)
    # rows of a part in vertex order
    for b in range(G):
        seg = perm[r["off"][b]:r["off"][b + 1]]
        assert np.all(np.diff(seg) > 0)


def test_permuted_system_is_PAPt_without_rounding_residue(harness, case):
    _, Q, A = case
    n = Q.shape[0]
    r = run(harness, Q, A, 8, 2, 4)
    perm = r["perm"]
    Pm = sp.csr_matrix((np.ones(n), (np.arange(n), perm)), shape=(n, n))
    ref = (Pm @ A @ Pm.T).tocsr()
    d = np.sqrt(np.abs(ref.diagonal()))
    C = ref.tocoo()
    rel = np.abs(C.data) / (d[C.row] * d[C.col])
    big = (rel > 1e-8) | (C.row == C.col)
    kept = sp.csr_matrix((C.data[big], (C.row[big], C.col[big])), shape=(n, n))
    got = r["Ap"]
    assert got.nnz == kept.nnz
    np.testing.assert_allclose(got.toarray()[kept.nonzero()], kept.data.astype(np.float32), rtol=0)
    assert abs(got - kept.astype(np.float32)).max() == 0.0
    # the dropped entries are cancellation residue: about half the row on a Kuhn grid
    assert (~big).sum() > 0.3 * (C.row != C.col).sum()
    assert rel[~big].max() < 1e-12
    np.testing.assert_allclose(r["dinv"], (1.0 / ref.diagonal()).astype(np.float32), rtol=1e-7)
    for v in range(0, n, max(1, n // 50)):                   # columns ascending per row
        assert np.all(np.diff(got.indices[got.indptr[v]:got.indptr[v + 1]]) > 0)


def test_local_table_is_the_symmetric_scaled_block_within_bf16(harness, case):
    _, Q, A = case
    r = run(harness, Q, A, 8, 2, 4)
    Ap = r["Ap"].astype(np.float64).toarray()
    dg = np.diag(Ap).copy()
    S = Ap / np.sqrt(np.outer(dg, dg))
    blocks = local_blocks(r)
    for b, O in enumerate(blocks):
        o0, o1 = r["off"][b], r["off"][b + 1]
        ref = S[o0:o1, o0:o1] - np.eye(o1 - o0)
        np.testing.assert_array_equal(O, O.T)                       # exactly symmetric
        np.testing.assert_allclose(O, ref, atol=2.0 ** -8 * np.abs(ref).max())
        # every in-part coupling is present (no row exceeds the width here)
        assert np.all((np.abs(ref) > 1e-6) == (O != 0.0))
        # Gershgorin bound covers the block's spectrum
        lam = np.linalg.eigvalsh(np.eye(o1 - o0) + O)
        assert lam.max() <= r["lmax"] + 1e-12 and lam.min() > 0


@pytest.mark.parametrize("degree", [2, 3, 4, 6])
def test_chebyshev_coefficients_match_the_closed_form(harness, case, degree):
    _, Q, A = case
    r = run(harness, Q, A, 8, 2, degree)
    lmax = r["lmax"]
    lmin = lmax / 30.0
    th, de = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    lam = np.linspace(1e-3, lmax, 257)
    # p(lambda) from the recurrence on the scalar "matrix" lambda
    x = r["c0"] * np.ones_like(lam)
    dk = x.copy()
    res = 1.0 - lam * x
    for i in range(1, degree):
        dk = r["c1"][i] * dk + r["c2"][i] * res
        x = x + dk
        res = res - lam * dk
    Tk = np.polynomial.chebyshev.Chebyshev.basis(degree)
    closed = 1.0 - Tk((th - lam) / de) / Tk(th / de)
    np.testing.assert_allclose(lam * x, closed, atol=2e-6)
    assert np.all(x > 0)                                      # positive on (0, lmax]


def test_preconditioner_is_spd_and_cuts_cg_iterations(harness, case):
    _, Q, A = case
    n = Q.shape[0]
    r = run(harness, Q, A, 8, 2, 4)
    Ap = r["Ap"].astype(np.float64)
    dinv = r["dinv"].astype(np.float64)
    blocks = local_blocks(r)

    def prec(y):
        out = np.empty_like(y)
        for b, O in enumerate(blocks):
            o0, o1 = r["off"][b], r["off"][b + 1]
            out[o0:o1] = cheb_apply(r, y[o0:o1], O, dinv[o0:o1])
        return out

    # SPD on one part, assembled column by column
    o0, o1 = r["off"][0], r["off"][1]
    Mb = np.stack([cheb_apply(r, e, blocks[0], dinv[o0:o1]) for e in np.eye(o1 - o0)], axis=1)
    np.testing.assert_allclose(Mb, Mb.T, atol=1e-6 * np.abs(Mb).max())
    assert np.linalg.eigvalsh(0.5 * (Mb + Mb.T)).min() > 0

    def pcg(M, b, tol=1e-6):
        x = np.zeros_like(b)
        rr = b.copy()
        u = M(rr)
        p = u.copy()
        g = rr @ u
        for it in range(5000):
            if np.linalg.norm(rr) <= tol * np.linalg.norm(b):
                return it
            s = Ap @ p
            al = g / (p @ s)
            x += al * p
            rr -= al * s
            u = M(rr)
            gn = rr @ u
            p = u + (gn / g) * p
            g = gn
        return 5000

    b = np.random.default_rng(0).standard_normal(n)
    it_j = pcg(lambda y: dinv * y, b)
    it_p = pcg(prec, b)
    assert it_p <= 0.6 * it_j, (it_p, it_j)


def test_sizes_that_do_not_fit_are_refused(harness, case):
    _, Q, A = case
    n = Q.shape[0]
    G = (n + 2 * NT - 1) // (2 * NT) - 1                      # one part too few for 2 rows per thread
    assert not run(harness, Q, A, G, 2, 4)["ok"]
    assert not run(harness, Q, A, 8, 2, 9)["ok"]              # degree above the maximum
    r = run(harness, Q, A, 8, 2, 1)                           # degree 1: Jacobi, no table
    assert r["ok"] and r["lw"] == 0 and r["loc"].size == 0
