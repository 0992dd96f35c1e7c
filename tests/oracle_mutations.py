"""Mutation sweep over the oracle: does every plausible one-token mistake in
oracle/ turn a CPU test red?

Each mutation below replaces one expression of the oracle (a sign, a factor,
a link offset, a conjugation, one step of an algorithm) by a plausible wrong
form.  The sweep copies oracle/ into a scratch mirror of the repository
(everything else symlinked), applies one mutation, runs the oracle's CPU
tests, and reports the mutants that no test catches.  Not collected by
pytest (it takes about a quarter of an hour); run it by hand:

    python tests/oracle_mutations.py [--workdir DIR] [index ...]

Exit status 1 if a mutant survives or a pattern is not found exactly once in
its file (a pattern that also matched a docstring would mutate the wrong
text).
"""

import argparse
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))

# (file in oracle/, exact text, replacement, the mistake it models)
MUTATIONS = [
    ("dirac.py", "g[-1] *= bc_t", "g[0] *= bc_t", "time-boundary sign on the wrong slice"),
    ("dirac.py", "fwd = spin_mul(eye - gammas[mu]", "fwd = spin_mul(eye + gammas[mu]", "forward projector sign"),
    ("dirac.py", "bwd = spin_mul(eye + gammas[mu]", "bwd = spin_mul(eye - gammas[mu]", "backward projector sign"),
    ("dirac.py", "ub = dag(link_at(umu, {mu: -1}))", "ub = dag(umu)", "backward hop with the site's own link"),
    ("dirac.py", "q2 = (un @ dag(link_at(um, {mu: -1, nu: 1}))", "q2 = (un @ link_at(um, {mu: -1, nu: 1})",
     "a clover leaf factor without its dagger"),
    ("dirac.py", "out.append((q - dag(q)) / 8.0)", "out.append((q - dag(q)) / 4.0)", "field-strength normalisation"),
    ("dirac.py", "out.append((q - dag(q)) / 8.0)", "out.append((q + dag(q)) / 8.0)", "Hermitian instead of anti-Hermitian part"),
    ("dirac.py", "c *= 1j * kappa * csw", "c *= 0.5j * kappa * csw", "clover prefactor halved"),
    ("dirac.py", "c *= 1j * kappa * csw", "c *= -1j * kappa * csw", "clover prefactor sign"),
    ("dirac.py", "sigma(gammas, mu, nu))\n    c *=", "sigma(gammas, nu, mu))\n    c *=", "sigma indices transposed"),
    ("dirac.py", "return x + site_mul(self.c, x) - self.kappa * self.hop(x)",
     "return x + site_mul(self.c, x) + self.kappa * self.hop(x)", "hopping-term sign in D"),
    ("dirac.py", "return x - self.kappa * site_mul(self.cinv, self.hop(x))",
     "return x + self.kappa * site_mul(self.cinv, self.hop(x))", "hopping-term sign in A"),
    ("dirac.py", "self.colour = sum(coords[mu] // domain[mu] for mu in range(4)) % 2",
     "self.colour = sum(coords[mu] // domain[mu] for mu in range(3)) % 2", "domain colouring without t"),
    ("dirac.py", "!= domain[mu] - 1).astype(float)", "!= domain[mu]).astype(float)", "intra-domain forward mask off by one"),
    ("dirac.py", "return pr * (-self.kappa * site_mul(self.cinv, h))",
     "return pr * (self.kappa * site_mul(self.cinv, h))", "sign of the off-diagonal SAP blocks"),
    ("dirac.py", "return np.linalg.inv(np.eye(12) + c)", "return np.linalg.inv(np.eye(12) - c)", "C_inv of 1 - C"),
    ("gamma.py", "return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])", "return 1.0j * (g[mu] @ g[nu] - g[nu] @ g[mu])",
     "sigma normalisation"),
    ("gamma.py", "g2 = np.array([[0, 0, 0, 1], [0, 0, -1, 0], [0, -1, 0, 0], [1, 0, 0, 0]])",
     "g2 = np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]])", "gamma_2 sign"),
    ("gamma.py", "return np.block([[i2, i2], [i2, -i2]])", "return np.block([[i2, -i2], [i2, i2]])", "chiral rotation"),
    ("sap.py", "    x = 2 * b - q", "    x = b - q", "first Jacobi step"),
    ("sap.py", "        x = x + b - q", "        x = x - b + q", "later Jacobi steps"),
    ("sap.py", "s = s + me * (b - q_e)", "s = s + me * (b + q_e)", "E residual update sign"),
    ("sap.py", "s = s - op.A_block(x_e, O, E)           # s_O", "s = s + op.A_block(x_e, O, E)           # s_O",
     "O source update sign"),
    ("sap.py", "s = s - op.A_block(x_o, E, O)", "s = s + op.A_block(x_o, E, O)", "E source update sign"),
    ("sap.py", "    return x_e + x_o\n", "    return x_e - x_o\n", "combination of the two colours"),
    ("sap.py", "    x_e = jacobi(op, s, E, n_jac)\n    s = s - op.A_block(x_e, O, E)\n",
     "    x_e = jacobi(op, s, E, n_jac)\n    s = s - 0.5 * op.A_block(x_e, O, E)\n", "closing sweep's coupling"),
    ("solvers.py", "beta = alpha * rho / (rho0 * omega)", "beta = rho / rho0", "Algorithm 5 beta"),
    ("solvers.py", "omega = vdot(t, r) / tt", "omega = vdot(r, t) / tt", "Algorithm 5 omega conjugated"),
    ("solvers.py", "alpha = rho0 / rtq", "alpha = rho0 / rtq.conjugate()", "Algorithm 5 alpha conjugated"),
    ("solvers.py", "p = r + beta * (p - omega * q)", "p = r + beta * (p + omega * q)", "Algorithm 5 direction update"),
    ("solvers.py", "rho = vdot(rt, r)\n        if record", "rho = vdot(r, rt)\n        if record", "Algorithm 5 rho conjugated"),
    ("solvers.py", "dx = err * (to_double(q) if single else q)", "dx = (to_double(q) if single else q)",
     "Algorithm 4 correction without the residual norm"),
    ("pointwise.py", "sf = bc_t if (mu == 3 and cf[3] == dims[3]) else 1.0", "sf = 1.0",
     "site-by-site D without the time-boundary sign"),
    ("pointwise.py", "@ (eye + gammas[mu]).T", "@ (eye - gammas[mu]).T", "site-by-site backward projector"),
    ("pointwise.py", "return (q - h(q)) / 8.0", "return (q - h(q)) / 4.0", "site-by-site field strength"),
    ("pointwise.py", "+ L(nu, 0, 0) @ h(L(mu, -1, 1))", "+ L(nu, 0, 0) @ L(mu, -1, 1)", "site-by-site clover leaf"),
    ("pointwise.py", "@ (eye - gammas[mu]).T", "@ (eye - gammas[mu])", "site-by-site projector transposed"),
    ("grad.py", "g[..., mu, :, :] = op.kappa * (g1 + g2)", "g[..., mu, :, :] = op.kappa * (g1 - g2)", "hopping force sign"),
    ("grad.py", "w = -1j * op.kappa * op.csw * z", "w = 1j * op.kappa * op.csw * z", "clover force sign"),
    ("grad.py", "v = (w - dag(w)) / 8.0", "v = (w - dag(w)) / 4.0", "clover force normalisation"),
    ("grad.py", "contrib = r if dg else dag(r)", "contrib = dag(r) if dg else r", "clover force dagger"),
    ("grad.py", "return a - tr[..., None, None] / 3.0 * np.eye(3)", "return a", "su(3) projection without the trace"),
    ("grad.py", "lf = shift_fwd(lam, mu, op.bc_t)", "lf = shift_fwd(lam, mu, 1)", "force without the time-boundary sign"),
]

TESTS = ["tests/test_oracle_dirac.py", "tests/test_oracle_gamma.py", "tests/test_oracle_grad.py",
         "tests/test_oracle_sap.py", "tests/test_oracle_solvers.py", "tests/test_oracle_flops.py"]


def mirror(workdir):
    """A copy of oracle/ with everything else of the repository symlinked."""
    if os.path.exists(workdir):
        shutil.rmtree(workdir)
    os.makedirs(workdir)
    for name in os.listdir(ROOT):
        if name in (".git", "oracle") or name.startswith("_"):
            continue
        os.symlink(os.path.join(ROOT, name), os.path.join(workdir, name))
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(workdir, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workdir", default=None, help="scratch mirror (default: a new temporary directory)")
    ap.add_argument("index", nargs="*", type=int, help="run only these mutations")
    args = ap.parse_args()
    workdir = args.workdir or os.path.join(tempfile.mkdtemp(prefix="oracle_mutations_"), "repo")
    bad = 0
    for i in args.index or range(len(MUTATIONS)):
        f, old, new, what = MUTATIONS[i]
        mirror(workdir)
        path = os.path.join(workdir, "oracle", f)
        src = open(path).read()
        if src.count(old) != 1:
            print(f"{i:2d} {f:12s} pattern found {src.count(old)} times: {what}", flush=True)
            bad += 1
            continue
        open(path, "w").write(src.replace(old, new))
        r = subprocess.run([sys.executable, "-m", "pytest", *TESTS, "-x", "-q", "-p", "no:cacheprovider"],
                           cwd=workdir, capture_output=True, text=True)
        caught = r.returncode != 0
        bad += 0 if caught else 1
        tail = [ln for ln in r.stdout.splitlines() if "passed" in ln or "failed" in ln][-1:]
        print(f"{i:2d} {f:12s} {'caught  ' if caught else 'SURVIVED'} {what}  ({tail[0] if tail else ''})",
              flush=True)
    shutil.rmtree(workdir, ignore_errors=True)
    print(f"{len(args.index or MUTATIONS) - bad} of {len(args.index or MUTATIONS)} mutations caught")
    sys.exit(1 if bad else 0)


if __name__ == "__main__":
    main()
