"""The bench's roofline arithmetic, on the CPU (no GPU, no library calls).

The headline line reports the default CTR kernel against three ceilings in
GB/s of plaintext: HBM at 2 bytes moved per plaintext byte, the shared-memory
pipe at the kernel's executed lookups per block, and the integer ALU pipe at
its ALU instructions per block (the INT32 term).  These checks pin that
arithmetic to the definitions, written out here independently, and check
that a summary whose source hash no longer matches the kernel is not used.
"""
import types

import pytest

import bench

PROBES = {"lds32": 32.0, "lop3": 64.0}
SMS, CLOCK_MHZ, HBM = 152, 2070.0, 6752.8


def args(**kw):
    a = dict(mode="ctr", bits=128, bpt=0, variant=0, size_mib=8192, cta=0)
    a.update(kw)
    return types.SimpleNamespace(**a)


def test_structural_lookup_count():
    """16 lookups per round from round 3 plus the final round, 5 for rounds
    1-2, and 15 per counter-run piece (one piece per run in whole waves, the
    last partial wave's runs split in 1, 2, 4 or 8 pieces so the busiest warp
    has the least to do there, each piece's setup counted as a quarter step)."""
    a = args()
    nbytes = 8 << 30
    runs = nbytes // 16 // 256
    warps = SMS * 32
    whole = runs - runs % warps
    tail = runs - whole
    # busiest warp's cost in quarter steps: 4 per step, 1 for each piece's setup
    busiest = {p: -(-tail * p // warps) * (4 * (8 // p) + 1) for p in (1, 2, 4, 8)}
    split = min(p for p in busiest if busiest[p] == min(busiest.values()))
    pieces = whole + tail * split
    want = 16 * 8 + 5 + 15 * pieces / (nbytes / 16)
    assert bench.executed_lookups_per_block(a, 128, nbytes, SMS) == pytest.approx(want, abs=1e-3)
    assert bench.executed_lookups_per_block(a, 256, nbytes, SMS) == pytest.approx(want + 64, abs=1e-3)
    # other modes and explicit block-per-thread shapes run the plain 16 * Nr
    assert bench.executed_lookups_per_block(args(mode="ecb_enc"), 192, nbytes, SMS) == 192
    assert bench.executed_lookups_per_block(args(bpt=2), 128, nbytes, SMS) == 160


def test_three_ceilings_and_the_binding_term():
    a = args()
    nbytes = 8 << 30
    per_launch_s = 7.8e-3
    rl = bench.roofline(a, 128, nbytes, per_launch_s, PROBES, SMS, CLOCK_MHZ, HBM, "measured")
    lk = rl["lookups_per_block_executed"]
    lds_peak = 32 * SMS * CLOCK_MHZ * 1e6  # lookups per second
    assert rl["peak"] == pytest.approx(lds_peak / 1e9, rel=1e-4)
    assert rl["achieved"] == pytest.approx(lk * nbytes / 16 / per_launch_s / 1e9, rel=1e-3)
    assert rl["frac"] == pytest.approx(rl["achieved"] / rl["peak"], rel=1e-3)
    terms = rl["ceilings_gbps_plaintext"]
    assert terms["hbm"] == pytest.approx(HBM / 2, rel=1e-4)
    assert terms["lds"] == pytest.approx(lds_peak / lk * 16 / 1e9, rel=1e-3)
    value = nbytes / per_launch_s / 1e9
    assert rl["binding"] == min(terms, key=terms.get)
    assert rl["frac_of_roofline"] == pytest.approx(value / terms[rl["binding"]], rel=1e-3)
    assert rl["analytic_ops_per_block"] == 160
    assert rl["hbm_frac"] == pytest.approx(2 * value / HBM, rel=1e-3)
    if "alu" in terms:  # the committed summary matches the kernel: the INT32 term is there
        alu = rl["int32"]["alu_instructions_per_block"]
        assert terms["alu"] == pytest.approx(64 * SMS * CLOCK_MHZ * 1e6 / alu * 16 / 1e9, rel=1e-3)
        assert rl["int32"]["frac"] == pytest.approx(value * 1e9 / 16 * alu / (64 * SMS * CLOCK_MHZ * 1e6), rel=1e-3)


def test_a_stale_summary_is_not_used(monkeypatch, tmp_path):
    """A summary whose recorded source hash differs from the kernel source
    gives no counters: the bench falls back to the structural count and
    reports no traffic and no INT32 term."""
    import os
    import shutil

    prof = os.path.join(bench.ROOT, "profiles", bench.PROFILE_OF_VARIANT[0][0])
    fake_root = tmp_path / "root"
    (fake_root / "profiles").mkdir(parents=True)
    src_dir = fake_root / "paper_1403_7295_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    shutil.copy(prof, fake_root / "profiles")
    for src in bench.PROFILE_OF_VARIANT[0][1]:
        (src_dir / src).write_text("// a different kernel source\n")
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    a = args()
    assert bench.read_profile_field(a, "lookups_per_block_measured:") is None
    assert bench.read_traffic(a) is None
    rl = bench.roofline(a, 128, 8 << 30, 7.8e-3, PROBES, SMS, CLOCK_MHZ, HBM, "measured")
    assert rl["lookups_source"].startswith("the kernel's own lookup count")
    assert "int32" not in rl and rl["traffic"] is None
