"""The oracle pins are strong enough: each planted mistake must fail them.

Every mutation is applied to a temporary copy of the oracle (on the CPU);
the pin tests then run against that copy in a subprocess and must fail.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "drop the father's weight": (
        "rows.append(Bw[tree.father[t]] @ side.E_ext[t].T)", "pass"),
    "drop the ancestor weight": (
        "rows.append(B_prev @ side.E_ext[t].T)", "pass"),
    "weights without sqrt(#T_t)": (
        "om = math.sqrt(tree.subtree_count[t]) / nrm if nrm > 0 else 0.0",
        "om = 1.0 / nrm if nrm > 0 else 0.0"),
    "threshold eps instead of eps/2": (
        "thr = (0.5 * eps) ** 2\n    tail = 0.0", "thr = (1.0 * eps) ** 2\n    tail = 0.0"),
    "no transfer commit": (
        "Fnew[side.root] = Rt[side.root] @ side.E_ext[side.root]",
        "Fnew[side.root] = side.basis.transfer[side.root]"),
    "transposed column factor": ("S_new[b] = Rt @ Sx @ Rs.T", "S_new[b] = Rt @ Sx @ Rs"),
    "other side's R-factor ignored": ("rows.append(om * (Ro @ Sx))", "rows.append(om * Sx)"),
    "nearfield not updated": ("N_new[b] = Z.N[b] + At @ Bs.T", "N_new[b] = Z.N[b]"),
    "leaf SVD without weights": ("M = Vh @ Bw[t].T", "M = Vh"),
    "extended transfer without the identity block": (
        "Ex[k:, kf:] = np.eye(self.u)", "Ex[k:, kf:] = 0.0 * np.eye(self.u)"),
    "leaf extension from the first rows of A": (
        "r0 = tree.offset[t] - off0\n                self.leaf_ext", "r0 = 0\n                self.leaf_ext"),
    "ancestor weights scaled by the subtree root's count": (
        "om = math.sqrt(tree.subtree_count[a]) / nrm if nrm > 0 else 0.0",
        "om = math.sqrt(tree.subtree_count[side.root]) / nrm if nrm > 0 else 0.0"),
    "weights normalised by the unchanged coupling": (
        "                nrm = block_norm(b)\n                om = math.sqrt(tree.subtree_count[t])",
        "                nrm = float(np.linalg.norm(Z.S[b]))\n                om = math.sqrt(tree.subtree_count[t])"),
    "tail measured in singular values, not their squares": (
        "while r > 0 and tail + sigma[r - 1] ** 2 <= thr:\n        tail += sigma[r - 1] ** 2",
        "while r > 0 and tail + sigma[r - 1] <= thr:\n        tail += sigma[r - 1]"),
    "one-sided coupling padded above instead of below": (
        "return np.vstack([S, np.zeros((u, l))])", "return np.vstack([np.zeros((u, l)), S])[:k + u]"),
    "new directions with the wrong sign at the leaves": (
        "self.leaf_ext[t] = np.hstack([basis.leaf[t], F[r0:r0 + tree.size[t], :]])",
        "self.leaf_ext[t] = np.hstack([basis.leaf[t], -F[r0:r0 + tree.size[t], :]])"),
}


def _pins_fail(tmp_path, module, before, after, test_files):
    """Plant `after` for `before` in a copy of oracle/<module> and run the
    pin files against the copy: True when they fail."""
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle")
    path = tmp_path / "oracle" / module
    src = path.read_text()
    assert src.count(before) == 1
    path.write_text(src.replace(before, after))
    env = dict(os.environ)
    env["PYTHONPATH"] = os.pathsep.join([str(tmp_path), ROOT, os.path.join(ROOT, "tests")])
    files = [os.path.join(ROOT, "tests", f) for f in test_files]
    code = ("import sys, pytest; sys.path.insert(0, %r); import oracle; "
            "assert oracle.__file__.startswith(%r); "
            "sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider'] + %r))"
            % (str(tmp_path), str(tmp_path), files))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=str(tmp_path),
                       env=env, timeout=600)
    return r.returncode != 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    before, after = MUTATIONS[name]
    failed, out = _pins_fail(tmp_path, "update.py", before, after, ["test_oracle_update.py"])
    assert failed, out


MATVEC_MUTATIONS = {
    "forward transformation without the transfer": (
        "acc = acc + W.transfer[c].T @ xh[c]", "acc = acc + xh[c][:W.rank[s]]"),
    "backward transformation transposed": (
        "yh[c] = yh[c] + V.transfer[c] @ yh[t]", "yh[c] = yh[c] + V.transfer[c].T @ yh[t]"),
    "coupling transposed": (
        "yh[bt.row[b]] = yh[bt.row[b]] + Z.S[b] @ xh[bt.col[b]]",
        "yh[bt.row[b]] = yh[bt.row[b]] + Z.S[b].T @ xh[bt.col[b]]"),
    "nearfield dropped": ("out[rt.offset[t]:rt.offset[t] + rt.size[t]] += Z.N[b] @", "_ = Z.N[b] @"),
    "nearfield applied to the row cluster's entries": (
        "@ X[ct.offset[s]:ct.offset[s] + ct.size[s]]", "@ X[ct.offset[t]:ct.offset[t] + ct.size[t]]"),
    "backward transformation sons first": (
        "    for t in range(rt.n_clusters):\n        for c in rt.sons[t]:",
        "    for t in reversed(range(rt.n_clusters)):\n        for c in rt.sons[t]:"),
    "beta term scaled by alpha": (
        "res = res + beta * (", "res = res + alpha * beta * ("),
}


@pytest.mark.parametrize("name", sorted(MATVEC_MUTATIONS))
def test_matvec_pins_catch_mutation(name, tmp_path):
    before, after = MATVEC_MUTATIONS[name]
    failed, out = _pins_fail(tmp_path, "matvec.py", before, after, ["test_oracle_matvec.py"])
    assert failed, out


TREE_MUTATIONS = {
    "ties go to the highest axis": ("if ext[a] > ext[axis]:", "if ext[a] >= ext[axis]:"),
    "points on the midpoint go to the first son": (
        "first = idx[pts[:, axis] < mid]\n            second = idx[~(pts[:, axis] < mid)]",
        "first = idx[pts[:, axis] <= mid]\n            second = idx[~(pts[:, axis] <= mid)]"),
    "admissibility by the smaller diameter": (
        "max(self.rows.diam(t), self.cols.diam(s))", "min(self.rows.diam(t), self.cols.diam(s))"),
    "subdivision of a block with one leaf cluster": (
        "elif self.rows.is_leaf(t) or self.cols.is_leaf(s):",
        "elif self.rows.is_leaf(t) and self.cols.is_leaf(s):"),
    "sons of a block in column-major order": (
        "for t1 in self.rows.sons[t]:\n                for s1 in self.cols.sons[s]:",
        "for s1 in self.cols.sons[s]:\n                for t1 in self.rows.sons[t]:"),
    "squared box distance": (
        "return math.sqrt(float(np.sum(gap ** 2)))", "return float(np.sum(gap ** 2))"),
    "#T_t without t itself": (
        "self.subtree_count[t] = 1 + sum(", "self.subtree_count[t] = 0 + sum("),
}


@pytest.mark.parametrize("name", sorted(TREE_MUTATIONS))
def test_tree_pins_catch_mutation(name, tmp_path):
    before, after = TREE_MUTATIONS[name]
    failed, out = _pins_fail(tmp_path, "tree.py", before, after, ["test_oracle_tree.py"])
    assert failed, out


H2_MUTATIONS = {
    "transfer transposed in the expansion": (
        "parts = [self.dense(s) @ self.transfer[s] for s in self.tree.sons[t]]",
        "parts = [self.dense(s) @ self.transfer[s].T for s in self.tree.sons[t]]"),
    "coupling transposed in the block": (
        "return self.V.dense(bt.row[b]) @ self.S[b] @ self.W.dense(bt.col[b]).T",
        "return self.V.dense(bt.row[b]) @ self.S[b].T @ self.W.dense(bt.col[b]).T"),
    "sons of a subdivided block at its corner": (
        "r0 = self.V.tree.offset[tc] - t_off", "r0 = 0 * (self.V.tree.offset[tc] - t_off)"),
    "leaf matrices read row by row": (
        "cb.leaf[t] = np.array(leaf_data[pos:pos + m * k]).reshape((m, k), order=\"F\")",
        "cb.leaf[t] = np.array(leaf_data[pos:pos + m * k]).reshape((m, k), order=\"C\")"),
    "couplings read row by row": (
        "self.S[b] = np.array(data[pos:pos + k * l]).reshape((k, l), order=\"F\")",
        "self.S[b] = np.array(data[pos:pos + k * l]).reshape((k, l), order=\"C\")"),
}


@pytest.mark.parametrize("name", sorted(H2_MUTATIONS))
def test_h2_pins_catch_mutation(name, tmp_path):
    before, after = H2_MUTATIONS[name]
    failed, out = _pins_fail(tmp_path, "h2.py", before, after,
                             ["test_oracle_h2.py", "test_oracle_update.py", "test_oracle_matvec.py"])
    assert failed, out


MARGIN_MUTATIONS = {
    "margin always reported as small": ("    return min(lo, hi)", "    return 0.0 * min(lo, hi)"),
    "next tail sum from the wrong singular value": (
        "tail_next = tail_r + float(sigma[r - 1] ** 2)",
        "tail_next = tail_r + float(sigma[min(r, len(sigma) - 1)] ** 2)"),
    "kept tail starts one value late": (
        "tail_r = float(np.sum(sigma[r:] ** 2))", "tail_r = float(np.sum(sigma[r + 1:] ** 2))"),
    "margin measured against eps/2 instead of its square": (
        "thr = (0.5 * eps) ** 2\n    tail_r", "thr = (0.5 * eps)\n    tail_r"),
}


@pytest.mark.parametrize("name", sorted(MARGIN_MUTATIONS))
def test_margin_pin_catches_mutation(name, tmp_path):
    before, after = MARGIN_MUTATIONS[name]
    failed, out = _pins_fail(tmp_path, "update.py", before, after, ["test_oracle_rank_margin.py"])
    assert failed, out


LR_MUTATIONS = {
    "Schur complement added instead of subtracted": (
        "_mul(C, -1.0, d21, d12, d22)", "_mul(C, 1.0, d21, d12, d22)"),
    "forward substitution without L21 X1": (
        "Y2 = Y[n1:] - Z.block_dense(_son(bt, d, t2, t1)) @ X1", "Y2 = Y[n1:]"),
    "backward substitution without R12 X2": (
        "Y1 = Y[:n1] - Z.block_dense(_son(bt, d, t1, t2)) @ X2", "Y1 = Y[:n1]"),
    "low-rank term with the coupling transposed": (
        'return ("lr", alpha * (Xt @ ZY.S[y]), ZY.W.dense(r))', 'return ("lr", alpha * (Xt @ ZY.S[y].T), ZY.W.dense(r))'),
    "low-rank term from the wrong factor's basis": (
        "Xt = ZX.block_dense(x) @ ZY.V.dense(s)", "Xt = ZX.block_dense(x) @ ZX.V.dense(s)"),
    "temporaries dropped": (
        'out.append(("temp", z, temps.get((t1, r1), [])))', 'out.append(("temp", z, []))'),
    "leaf LU without the division by the pivot": ("A[k + 1:, k] /= A[k, k]", "A[k + 1:, k] *= 1.0"),
    "right solve with the unit lower factor": (
        'return solve_triangular(Z.N[d], Y.T, trans="T", lower=False).T',
        'return solve_triangular(Z.N[d], Y.T, trans="T", lower=True, unit_diagonal=True).T'),
    "forward substitution on an admissible leaf keeps the old coupling": (
        "Ws = Z.W.dense(s)\n        Z.S[x] = np.zeros_like(Z.S[x])", "Ws = Z.W.dense(s)"),
    "conjugate directions not conjugated": ("p = z + (rz_new / rz) * p", "p = z.copy()"),
    "rank cap not passed to the local update": (
        "C.eps, max_rank=C.rank_cap)", "C.eps, max_rank=None)"),
}


@pytest.mark.parametrize("name", sorted(LR_MUTATIONS))
def test_lr_pins_catch_mutation(name, tmp_path):
    before, after = LR_MUTATIONS[name]
    failed, out = _pins_fail(tmp_path, "lr.py", before, after, ["test_oracle_lr.py"])
    assert failed, out


INVERSE_MUTATIONS = {
    "off-diagonal block of the inverse with the wrong sign": (
        "mul(Cm, T, Cm, -1.0, d12, d22, d12, C.eps, C.cap, C.rank_cap)",
        "mul(Cm, T, Cm, 1.0, d12, d22, d12, C.eps, C.cap, C.rank_cap)"),
    "C11 without the correction C12 B21": (
        "    C.updates += mul(Cm, Cm, T, -1.0, d12, d21, d11, C.eps, C.cap, C.rank_cap)  # C11 = C11 - C12 B21\n", ""),
    "Schur complement without the product A21 B12": (
        "mul(A, A, T, -1.0, d21, d12, d22, C.eps, C.cap, C.rank_cap)", "0"),
    "leaf inverse without the backward solve": (
        "return solve_triangular(F, Y, lower=False)", "return Y"),
}


@pytest.mark.parametrize("name", sorted(INVERSE_MUTATIONS))
def test_inverse_pins_catch_mutation(name, tmp_path):
    before, after = INVERSE_MUTATIONS[name]
    failed, out = _pins_fail(tmp_path, "lr.py", before, after, ["test_oracle_inverse.py"])
    assert failed, out


FEM_MUTATIONS = {
    "element entries up to 60% of the diagonal taken for noise": (
        "Ke[np.abs(Ke) <= 1e-12 * np.abs(np.diag(Ke)).max()] = 0.0",
        "Ke[np.abs(Ke) <= 0.6 * np.abs(np.diag(Ke)).max()] = 0.0"),
    "element matrix without the coefficient": (
        "Ke = sigma[flat] * vol * (G @ G.T)", "Ke = vol * (G @ G.T)"),
}


@pytest.mark.parametrize("name", sorted(FEM_MUTATIONS))
def test_fem_pins_catch_mutation(name, tmp_path):
    before, after = FEM_MUTATIONS[name]
    failed, out = _pins_fail(tmp_path, "fem.py", before, after, ["test_oracle_fem.py"])
    assert failed, out


CHOL_MUTATIONS = {
    "Schur complement of the Cholesky added instead of subtracted": (
        "_mul_t(C, -1.0, d21, d21, d22, lower=True)", "_mul_t(C, 1.0, d21, d21, d22, lower=True)"),
    "right solve without the X1 L21^* term": (
        "        _mul_t(C, -1.0, _son(bt, x, t1, s1), _son(bt, d, s2, s1), _son(bt, x, t1, s2), lower=False)\n",
        "        pass\n"),
    "transposed admissible factor with its coupling not transposed": (
        'return ("lr", alpha * (Xt @ Z.S[yh].T), Z.V.dense(r))', 'return ("lr", alpha * (Xt @ Z.S[yh]), Z.V.dense(r))'),
    "diagonal target computing the blocks above the diagonal instead of below": (
        "tree.offset[t1] < tree.offset[r1]", "tree.offset[t1] > tree.offset[r1]"),
    "leaf Cholesky without the square root of the pivot": ("A[k, k] = np.sqrt(d)", "A[k, k] = d"),
    "backward solve reading the upper block instead of the factor's transpose": (
        "Y1 = Y[:n1] - Z.block_dense(_son(bt, d, t2, t1)).T @ X2",
        "Y1 = Y[:n1] - Z.block_dense(_son(bt, d, t1, t2)) @ X2"),
}


@pytest.mark.parametrize("name", sorted(CHOL_MUTATIONS))
def test_chol_pins_catch_mutation(name, tmp_path):
    before, after = CHOL_MUTATIONS[name]
    failed, out = _pins_fail(tmp_path, "chol.py", before, after, ["test_oracle_chol.py"])
    assert failed, out
