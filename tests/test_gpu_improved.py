"""GPU parity of the static improved estimator (Sec. 2.4, Eq.
PImprovedEstimatorStatic) through the C ABI: the traces of the sequences
with one annihilator replaced by its Bulla operator [c_f, U]
(ctq_add_bulla_operators, ctq_eval_traces) and the ratios h^st = w^U / w
(ctq_static_ratios), against oracle.improved.

Bars: each replaced trace as any FP64 trace (relative 1e-12, or 8x the
chain's own float64 rounding spread; two-float: the two-float bar); the
ratio kernel against the same arithmetic on the host to 16 ulps (the
device and host exponentials and complex products round differently); h^st
against the oracle's ratio within the two traces' bars propagated through
the quotient."""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity  # noqa: E402
from oracle import atom  # noqa: E402
from oracle import improved as OI  # noqa: E402
from paper_2010_08482_gb300 import ctq  # noqa: E402
from paper_2010_08482_gb300 import workloads as w  # noqa: E402

pytestmark = pytest.mark.gpu

X2_REL = 100.0 * parity.FP64_REL
STATED_TC = {(ctq.TF32X3, "t2g"): 1e-4}  # 5x the 3xTF32 bar of plain t2g traces (one operator replaced)


def small_complex_model():
    cf = w.crystal_field_complex(4, 0.3, 17)
    return w.ModelParams("k2c", n_orb=2, l=0, interaction="kanamori", U=3.0, J=0.6, beta=4.0, mu=1.1,
                         n0=2, cf=cf, sector_mode="n")


def evaluate(imp, sub, n_flav, precision=ctq.FP64):
    bu, chain, pos = w.bulla_sequences(sub, n_flav)
    db, dbu = ctq.DeviceBatch(sub), ctq.DeviceBatch(bu)
    ev = ctq.StaticImprovedEvaluator(imp, sub.n_chains, bu.n_chains, max(db.max_ops, 1), precision=precision)
    ch = torch.as_tensor(chain, device="cuda")
    ev(db, dbu, ch)
    torch.cuda.synchronize()
    return bu, chain, pos, ev


def log_scale(ref, kind):
    return parity.log_sum_abs_q0(ref) if kind == "sum_q0" else ref["log_abs"]


# The conditioning-scale allowance (floor x e^{log_cond - log scale}) never
# exceeds this relative error, and the entries that pass only because of it
# are counted.
FLOOR_CAP = 1e-8
# Absolute allowance on a one-pass ratio h^st (energy units of the model,
# |h| ~ U): a replaced trace that nearly cancels (|w^U| << |w|) carries the
# float64 rounding of terms of the size of w, about 1e-15 |w|, which is a
# large relative error of a tiny h; entries that need it are counted.
H_ABS = 1e-13


class FloorCount:
    """Entries whose error exceeds their arithmetic bar and pass only because
    of the (capped) conditioning-scale or absolute allowance; check() prints
    the count and asserts at most max(3, 10 %) of the entries seen."""

    def __init__(self, label):
        self.label, self.n, self.hits = label, 0, []

    def bar(self, err, base, allowed, key):
        """base: the arithmetic bar; allowed: the bar including the capped
        conditioning allowance.  Returns max(base, allowed)."""
        self.n += 1
        allowed = max(base, allowed)
        if err > base:
            self.hits.append((key, err, base, allowed))
        return allowed

    def check(self):
        lim = max(parity.WIDEN_MIN, int(parity.WIDEN_FRAC * self.n))
        for key, err, base, allowed in self.hits[:20]:
            print(f"{self.label}: entry {key} err {err:.2e} above its arithmetic bar {base:.2e}, "
                  f"within the conditioning allowance {allowed:.2e}")
        print(f"{self.label}: {len(self.hits)} of {self.n} entries pass only on the conditioning allowance "
              f"(allowed {lim})")
        assert len(self.hits) <= lim, (self.label, len(self.hits), self.n)


def check(m, mb, sub, bu, chain, ev, bar, scale_floor=0.0, label="h^st", floor_cap=FLOOR_CAP):
    """Replaced traces and ratios against the oracle; returns the worst errors.
    bar(key, ref, err) gives a trace's arithmetic bar (a parity.Bars method,
    which counts widened chains; err lets a mixed bar count only the chains
    that needed the widening).  scale_floor > 0 (two different eigenbases) also
    allows that much error relative to the configuration's conditioning scale
    e^{log_cond} (the float64 rounding of the two bases' blocks, which a
    near-cancelling trace does not scale down), at most floor_cap, with the
    entries that need it counted (FloorCount)."""
    floors = FloorCount(label)
    n_seq = bu.n_chains
    ru = ev.repl.results(n_seq)
    rb = ev.base.results(sub.n_chains)
    ref_u = parity.oracle_chain_results(mb, bu, range(n_seq))
    ref_b = parity.oracle_chain_results(mb, sub, range(sub.n_chains))
    h = ev.ratios(n_seq)
    worst_u = worst_h = 0.0
    for i in range(n_seq):
        c = int(chain[i])
        rw = ref_b[c]
        if ref_u[i]["log_abs"] == -math.inf and ru["log_abs"][i] != -math.inf:
            # exactly zero in the oracle (a symmetry of its eigenbasis):
            # float64 rounding noise only, far below the configuration's scale
            assert rw["log_cond"] != -math.inf and ru["log_abs"][i] < rw["log_cond"] - 20, (i, c)
            eu, ku, tu = 0.0, "zero", 0.0
        else:
            eu, ku = parity.chain_error(ru["log_abs"][i], ru["phase"][i], ref_u[i])
            tu = bar(i, ref_u[i], eu)
            if scale_floor > 0.0 and ref_u[i]["log_abs"] != -math.inf:
                lc = max(ref_u[i]["log_cond"], rw["log_cond"])
                tu = floors.bar(eu, tu, min(floor_cap, scale_floor * math.exp(lc - log_scale(ref_u[i], ku))),
                                ("w^U", i))
            assert eu <= tu, (i, c, eu, ku)
        worst_u = max(worst_u, eu)
        # the ratio kernel: the same quotient taken on the host from the
        # library's own two results
        la, lu = rb["log_abs"][c], ru["log_abs"][i]
        if not np.isfinite(la):
            assert math.isnan(h[i].real) and math.isnan(h[i].imag)
            continue
        if lu == -math.inf:
            assert h[i] == 0
        else:
            pu = complex(*ru["phase"][i])
            pb = complex(*rb["phase"][c])
            hh = math.exp(lu - la) * pu * pb.conjugate()
            assert abs(h[i] - hh) <= 16 * 2.0 ** -52 * abs(hh) + 1e-300, (i, h[i], hh)
        # against the oracle's ratio: bars of both traces through the quotient
        if rw["log_abs"] == -math.inf:
            continue
        ew, kw = parity.chain_error(la, rb["phase"][c], rw)
        tw = bar(c, rw, ew)
        if scale_floor > 0.0:
            tw = floors.bar(ew, tw, min(floor_cap, scale_floor * math.exp(rw["log_cond"] - log_scale(rw, kw))),
                            ("w", i))
        assert ew <= tw
        if ref_u[i]["log_abs"] == -math.inf:
            h_ref, su = 0j, math.exp(rw["log_cond"] - 20 - rw["log_abs"])
            tu = 1.0
        else:
            h_ref = (complex(ref_u[i]["phase"]) / complex(rw["phase"])
                     * math.exp(ref_u[i]["log_abs"] - rw["log_abs"]))
            su = math.exp(log_scale(ref_u[i], ku) - rw["log_abs"])
        sw = math.exp(log_scale(rw, kw) - rw["log_abs"])
        tol = 2.0 * (tu * su + tw * sw * abs(h_ref)) + 1e-300
        assert abs(h[i] - h_ref) <= tol, (i, c, h[i], h_ref, tol)
        if h_ref != 0:
            worst_h = max(worst_h, abs(h[i] - h_ref) / abs(h_ref))
    floors.check()
    return worst_u, worst_h


@pytest.mark.parametrize("name,n", [("hubbard2", 32), ("t2g", 48), ("d5", 4)])
def test_static_improved_fp64_on_oracle_eigenbasis(name, n, models):
    m = models(name)
    mb = OI.with_bulla(m)
    sub = w.WORKLOADS[name][1]().subset(range(n))
    imp = parity.load_oracle_model(ctq, m)
    imp.add_bulla_operators(atom.one_body_matrix(m.params, m.mu))
    assert imp.n_alpha == 3 * m.n_flav
    bu, chain, pos, ev = evaluate(imp, sub, m.n_flav)
    assert bu.n_chains > n
    bars = parity.Bars(f"{name} h^st fp64")
    wu, wh = check(m, mb, sub, bu, chain, ev, bars.fp64, label=f"{name} h^st fp64")
    bars.check()
    print(f"\n{name}: {bu.n_chains} replaced sequences, max rel err w^U {wu:.2e}, h^st {wh:.2e}")


@pytest.mark.parametrize("name", ["hubbard2", "complex"])
def test_static_improved_on_library_eigenbasis(name, models):
    """The library's own eigenbasis and one-body matrix (ctq_build_impurity,
    then ctq_add_bulla_operators with no matrix): traces and ratios are
    basis-invariant, so they compare with the oracle directly."""
    m = atom.Model(small_complex_model()) if name == "complex" else models(name)
    mb = OI.with_bulla(m)
    rng = np.random.default_rng(31)
    sub = w.random_batch(rng, m.n_flav, m.beta, 24, 2, 10)
    imp = ctq.build_impurity(m.params, device=0)
    imp.add_bulla_operators()
    bu, chain, pos, ev = evaluate(imp, sub, m.n_flav)

    bars = parity.Bars(f"{name} h^st library eigenbasis")

    def bar(key, ref, err=None):  # two eigenbases: 1e-11, or their float64 spread as well
        return bars.fp64(key, ref, base=1e-11)
    # two independent eigensolvers agree to ~1e-12 of the configuration's
    # scale, so a replaced trace 1e4 times below that scale carries ~1e-8
    wu, wh = check(m, mb, sub, bu, chain, ev, bar, scale_floor=1e-12, label=f"{name} h^st library eigenbasis",
                   floor_cap=1e-7)
    bars.check()
    print(f"\n{name} (library eigenbasis): max rel err w^U {wu:.2e}, h^st {wh:.2e}")


def test_static_improved_two_float(models):
    m = models("t2g")
    mb = OI.with_bulla(m)
    sub = w.WORKLOADS["t2g"][1]().subset(range(32))
    imp = parity.load_oracle_model(ctq, m)
    imp.add_bulla_operators(atom.one_body_matrix(m.params, m.mu))
    bu, chain, pos, ev = evaluate(imp, sub, m.n_flav, precision=ctq.F32X2)

    bars = parity.Bars("t2g h^st F32X2")

    def bar(key, ref, err=None):
        return bars.fp64(key, ref, base=X2_REL / 32.0, scale=32.0)
    wu, wh = check(m, mb, sub, bu, chain, ev, bar, label="t2g h^st F32X2")
    bars.check()
    print(f"\nt2g F32X2: max rel err w^U {wu:.2e}, h^st {wh:.2e}")


def test_static_improved_tensor_cores(models):
    m = models("t2g")
    mb = OI.with_bulla(m)
    sub = w.WORKLOADS["t2g"][1]().subset(range(24))
    imp = parity.load_oracle_model(ctq, m)
    imp.add_bulla_operators(atom.one_body_matrix(m.params, m.mu))
    assert ctq.trace_kernel(imp, ctq.TF32X3) == ctq.KERNEL_TC_SMALL
    bu, chain, pos, ev = evaluate(imp, sub, m.n_flav, precision=ctq.TF32X3)

    bars = parity.Bars("t2g h^st TF32X3")

    def bar(key, ref, err=None):
        return bars.mixed(key, ref, STATED_TC[(ctq.TF32X3, "t2g")], parity.UNIT[ctq.TF32X3], err)
    wu, wh = check(m, mb, sub, bu, chain, ev, bar, label="t2g h^st TF32X3")
    bars.check()
    print(f"\nt2g TF32X3: max rel err w^U {wu:.2e}, h^st {wh:.2e}")


def test_full_t2g_batch_sampled(models):
    """Every annihilator of the full 4096-chain t2g batch in one evaluation
    (the benchmark shape); sampled sequences against the oracle."""
    m = models("t2g")
    mb = OI.with_bulla(m)
    b = w.WORKLOADS["t2g"][1]()
    imp = parity.load_oracle_model(ctq, m)
    imp.add_bulla_operators(atom.one_body_matrix(m.params, m.mu))
    bu, chain, pos, ev = evaluate(imp, b, m.n_flav)
    h = ev.ratios(bu.n_chains)
    ru = ev.repl.results(bu.n_chains)
    assert np.all(np.isin(ru["status"], [ctq.CHAIN_OK, ctq.CHAIN_ZERO]))
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(bu.n_chains, size=48, replace=False))
    for i in sample:
        c = int(chain[i])
        tau, ops = b.chain(c)
        ratios = dict(OI.static_ratios(mb, tau, ops, beta=b.beta))
        h_ref = ratios[int(pos[i])]
        if math.isnan(h_ref.real):
            assert math.isnan(h[i].real)
            continue
        assert abs(h[i] - h_ref) <= 1e-9 * max(1.0, abs(h_ref)), (i, h[i], h_ref)


def test_ratio_kernel_edge_cases():
    """Zero, failed and out-of-range configurations; w^U = 0; complex phases."""
    dev = "cuda"
    la = torch.tensor([0.5, -math.inf, math.nan, 700.0], dtype=torch.float64, device=dev)
    ph = torch.tensor([1.0, 0.0, -1.0, 0.0, 0.0, 0.0, 0.6, 0.8], dtype=torch.float64, device=dev)
    chain = torch.tensor([0, 1, 2, 4, -1, 0, 3, 0], dtype=torch.int32, device=dev)
    lu = torch.tensor([1.25, 0.0, 0.0, 0.0, 0.0, -math.inf, 702.0, math.nan], dtype=torch.float64, device=dev)
    pu = torch.tensor([0.0, 1.0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, -0.8, 0.6, 1, 0], dtype=torch.float64, device=dev)
    out = torch.full((16,), 7.0, dtype=torch.float64, device=dev)
    ctq.static_ratios(chain, 4, la, ph, lu, pu, out)
    torch.cuda.synchronize()
    h = out.cpu().numpy()
    h = h[0::2] + 1j * h[1::2]
    assert abs(h[0] - math.exp(0.75) * 1j) <= 8 * 2.0 ** -52 * math.exp(0.75)
    for i in (1, 2, 3, 4, 7):  # w = 0, w failed, index out of range (twice), w^U failed
        assert math.isnan(h[i].real) and math.isnan(h[i].imag), i
    assert h[5] == 0
    ref6 = math.exp(2.0) * complex(-0.8, 0.6) * complex(0.6, -0.8)
    assert abs(h[6] - ref6) <= 16 * 2.0 ** -52 * abs(ref6)
    ctq.static_ratios(chain[:0], 4, la, ph, lu, pu, out)  # m = 0 launches nothing


# ---------------------------------------------------------------- one-pass ratios (ctq_eval_static_ratios)

def kind_of(ref):
    """The scale chain_error measures against: |w|, or sum_q0 |w_q0| when the
    q0 terms cancel."""
    return "sum_q0" if parity.log_sum_abs_q0(ref) - ref["log_abs"] > math.log(parity.CANCEL) else "abs"


def fused(imp, sub):
    db = ctq.DeviceBatch(sub)
    fe = ctq.FusedStaticEvaluator(imp, sub.n_chains, max(db.max_ops, 1), db.n_ops)
    fe(db)
    torch.cuda.synchronize()
    return fe.ratios(db.n_ops), fe.status.cpu().numpy()


def check_fused(m, mb, sub, hf, status, bar, floor, label="one pass", chains=None):
    """One-pass ratios against the oracle's ratio of every annihilator; every
    other entry exactly 0.  bar(key, ref): a trace's arithmetic bar (counted
    by a parity.Bars).  floor: error allowed relative to the replaced trace's
    conditioning scale e^{log_cond} (the one-pass product associates
    Y (Q (P A)) instead of the string order), at most FLOOR_CAP relative,
    or H_ABS absolute on h, with the entries that pass only on these
    allowances counted (FloorCount).  chains:
    the configurations to compare (default: all)."""
    bu, chain, pos = w.bulla_sequences(sub, m.n_flav)
    keep = np.arange(bu.n_chains) if chains is None else np.nonzero(np.isin(chain, chains))[0]
    floors = FloorCount(label)
    ref_u = parity.oracle_chain_results(mb, bu, keep)
    ref_b = parity.oracle_chain_results(mb, sub, np.unique(chain[keep]))
    ann = np.zeros(len(sub.op), bool)
    ann[np.asarray(sub.offsets[chain], np.int64) + pos] = True
    assert np.all(hf[~ann] == 0)
    worst = 0.0
    for i in keep:
        c = int(chain[i])
        k = int(sub.offsets[c]) + int(pos[i])
        rw, ru = ref_b[c], ref_u[i]
        if status[c] != ctq.CHAIN_OK:
            assert hf[k] == 0 and rw["log_abs"] == -math.inf
            continue
        if rw["log_abs"] == -math.inf:  # exactly zero in the oracle: the ratio is undefined
            continue
        if ru["log_abs"] == -math.inf:
            assert abs(hf[k]) <= 2 * floor * math.exp(rw["log_cond"] - rw["log_abs"]) + 1e-300, (i, hf[k])
            continue
        h_ref = complex(ru["phase"]) / complex(rw["phase"]) * math.exp(ru["log_abs"] - rw["log_abs"])
        ls_u = log_scale(ru, kind_of(ru))
        su = math.exp(ls_u - rw["log_abs"])
        sw = math.exp(log_scale(rw, kind_of(rw)) - rw["log_abs"])
        # both traces' bars carried through the quotient: arithmetic bars, and
        # the conditioning allowance (each term capped at FLOOR_CAP)
        tu, tw = bar(i, ru), bar(c, rw)
        fu = min(FLOOR_CAP, floor * math.exp(max(ru["log_cond"], rw["log_cond"]) - ls_u))
        fw = min(FLOOR_CAP, floor * math.exp(rw["log_cond"] - rw["log_abs"]))
        err = abs(hf[k] - h_ref)
        tol_base = 2.0 * (tu * su + tw * sw * abs(h_ref)) + 1e-300
        allowed = max(2.0 * (max(tu, fu) * su + max(tw, fw) * sw * abs(h_ref)), H_ABS)
        tol = floors.bar(err, tol_base, allowed, int(i))
        assert err <= tol, (i, c, int(pos[i]), hf[k], h_ref, tol)
        worst = max(worst, abs(hf[k] - h_ref) / abs(h_ref))
    floors.check()
    return worst


@pytest.mark.parametrize("name,n", [("hubbard2", 32), ("t2g", 48), ("d5", 4)])
def test_one_pass_ratios_on_oracle_eigenbasis(name, n, models):
    m = models(name)
    mb = OI.with_bulla(m)
    sub = w.WORKLOADS[name][1]().subset(range(n))
    imp = parity.load_oracle_model(ctq, m)
    imp.add_bulla_operators(atom.one_body_matrix(m.params, m.mu))
    hf, status = fused(imp, sub)
    bars = parity.Bars(f"{name} one pass")
    worst = check_fused(m, mb, sub, hf, status, bars.fp64, 1e-13, label=f"{name} one pass")
    bars.check()
    print(f"\n{name} one pass: max rel err h^st {worst:.2e}")


def test_one_pass_ratios_full_d5_batch_sampled(models):
    """The whole 1024-chain d5 batch in one pass (the benchmark shape); a
    seeded sample of 24 configurations (about 1,400 ratios) against the
    oracle."""
    m = models("d5")
    mb = OI.with_bulla(m)
    b = w.WORKLOADS["d5"][1]()
    imp = parity.load_oracle_model(ctq, m)
    imp.add_bulla_operators(atom.one_body_matrix(m.params, m.mu))
    hf, status = fused(imp, b)
    sample = np.sort(np.random.default_rng(23).choice(b.n_chains, size=24, replace=False))
    bars = parity.Bars("d5 one pass, full batch")
    worst = check_fused(m, mb, b, hf, status, bars.fp64, 1e-13, label="d5 one pass, full batch", chains=sample)
    bars.check()
    print(f"\nd5 one pass, full batch, 24 sampled configurations: max rel err h^st {worst:.2e}")


def dead_backward_cases():
    """t2g configurations whose backward product dies for one starting sector
    (tests/golden/t2g_dead_backward.json)."""
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "t2g_dead_backward.json")) as f:
        return [(c["tau"], c["op"]) for c in json.load(f)["chains"]]


def test_one_pass_ratios_when_a_backward_product_dies(models):
    """The one-pass kernel stops a string's backward pass when its product is
    exactly zero; the ratios of the earlier annihilators must still equal the
    oracle's (their other starting sectors carry them)."""
    m = models("t2g")
    mb = OI.with_bulla(m)
    chains = [(np.asarray(t, np.float64), np.asarray(o, np.int32)) for t, o in dead_backward_cases()]
    offs = np.cumsum([0] + [len(o) for _, o in chains]).astype(np.int32)
    sub = w.Batch(beta=m.beta, offsets=offs, tau=np.concatenate([t for t, _ in chains]),
                  op=np.concatenate([o for _, o in chains]))
    imp = parity.load_oracle_model(ctq, m)
    imp.add_bulla_operators(atom.one_body_matrix(m.params, m.mu))
    hf, status = fused(imp, sub)
    assert np.all(status == ctq.CHAIN_OK)
    bars = parity.Bars("t2g one pass, dead backward products")
    check_fused(m, mb, sub, hf, status, bars.fp64, 1e-13, label="t2g one pass, dead backward products")
    bars.check()
    for c, (tau, ops) in enumerate(chains):
        for pos, h_ref in OI.static_ratios(mb, tau, ops, beta=m.beta):
            got = hf[int(offs[c]) + pos]
            assert abs(got - h_ref) <= 1e-10 * max(1.0, abs(h_ref)), (c, pos, got, h_ref)


def test_one_pass_ratios_complex_library_eigenbasis(models):
    m = atom.Model(small_complex_model())
    mb = OI.with_bulla(m)
    rng = np.random.default_rng(31)
    sub = w.random_batch(rng, m.n_flav, m.beta, 24, 2, 10)
    imp = ctq.build_impurity(m.params, device=0)
    imp.add_bulla_operators()
    hf, status = fused(imp, sub)

    bars = parity.Bars("complex one pass, library eigenbasis")

    def bar(key, ref):
        return bars.fp64(key, ref, base=1e-11)
    worst = check_fused(m, mb, sub, hf, status, bar, 1e-12, label="complex one pass, library eigenbasis")
    bars.check()
    print(f"\ncomplex one pass (library eigenbasis): max rel err h^st {worst:.2e}")


def test_one_pass_needs_bulla_operators(models):
    m = models("hubbard2")
    imp = parity.load_oracle_model(ctq, m)
    with pytest.raises(ValueError):
        ctq.FusedStaticEvaluator(imp, 4, 8, 32)
