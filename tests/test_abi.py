"""Host-side checks of the C-ABI library (no GPU work): it loads, exports every
declared entry point, rejects bad arguments before any launch, and its paper
primitives (FindSeqSchedule, FitRanks, the plan's work units) agree with the
oracle's independent searches and the pebble-game simulator."""
import math
import os
import random
import re

import pytest

from oracle import bounds, pebble

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_09606_gb300 import build as b
    b.build()
    from paper_1908_09606_gb300 import cosma
    return cosma


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(cosma_[a-z0-9_]+)\s*\(", text))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    assert len(declared) >= 14
    raw = lib.load()
    for name in declared:
        assert hasattr(raw, name), f"{name} declared but not exported"
    bound = {s[0] for s in lib.SIGNATURES}
    assert declared == bound, f"binding out of sync: {declared ^ bound}"


def test_status_strings(lib):
    for s in range(-6, 1):
        assert lib.status_string(s) not in ("", "unknown status")


def test_rejects_bad_arguments_without_launch(lib):
    # negative sizes, short leading dimensions, null pointers, bad dtype
    assert lib.cosma_gemm(-1, 4, 4, 0, 4, 0, 4, 0, 4, lib.COSMA_F64) == lib.COSMA_ERR_INVALID_ARG
    assert lib.cosma_gemm(4, 4, 4, 0, 3, 0, 4, 0, 4, lib.COSMA_F64) == lib.COSMA_ERR_INVALID_ARG
    assert lib.cosma_gemm(4, 4, 4, 0, 4, 0, 3, 0, 4, lib.COSMA_F64) == lib.COSMA_ERR_INVALID_ARG
    assert lib.cosma_gemm(4, 4, 4, 0, 4, 0, 4, 0, 2, lib.COSMA_F64) == lib.COSMA_ERR_INVALID_ARG
    assert lib.cosma_gemm(4, 4, 4, 0, 4, 0, 4, 0, 4, lib.COSMA_F64) == lib.COSMA_ERR_INVALID_ARG
    assert lib.cosma_gemm(4, 4, 4, 8, 4, 8, 4, 8, 4, 9) == lib.COSMA_ERR_INVALID_ARG
    # host (non-device) pointers are refused before any launch
    import numpy as np
    a = np.zeros(16)
    p = a.ctypes.data
    assert lib.cosma_gemm(4, 4, 4, p, 4, p, 4, p, 4, lib.COSMA_F64) == lib.COSMA_ERR_INVALID_ARG
    # empty products are no-ops
    assert lib.cosma_gemm(0, 4, 4, 0, 4, 0, 4, 0, 4, lib.COSMA_F64) == lib.COSMA_OK
    assert lib.cosma_gemm(4, 0, 4, 0, 4, 0, 1, 0, 1, lib.COSMA_F64) == lib.COSMA_OK
    assert lib.cosma_gemm_grouped([], lib.COSMA_F32) == lib.COSMA_OK
    assert lib.cosma_gemm_grouped([], lib.COSMA_F64) == lib.COSMA_ERR_UNSUPPORTED


def test_k_limits_are_refused_before_any_launch(lib):
    # 65535 k blocks of 32 is the longest k; one more element is unsupported,
    # decided before the pointers are even looked at
    kmax = 65535 * 32
    dt = lib.COSMA_F32_EMU_TF32
    assert lib.cosma_gemm(4, 4, kmax + 1, 16, kmax + 1, 16, 4, 16, 4, dt) == \
        lib.COSMA_ERR_UNSUPPORTED
    assert lib.cosma_gemm(4, 4, kmax, 16, kmax, 16, 4, 16, 4, dt) == lib.COSMA_ERR_INVALID_ARG
    assert lib.cosma_gemm(4, 4, kmax + 1, 16, kmax + 1, 16, 4, 16, 4, lib.COSMA_F32) == \
        lib.COSMA_ERR_INVALID_ARG
    # the emulated path: 1023 slice panels of 2048
    emax = 1023 * 2048
    dt = lib.COSMA_F64_EMU_BF16
    assert lib.cosma_gemm(4, 4, emax + 1, 16, emax + 1, 16, 4, 16, 4, dt) == \
        lib.COSMA_ERR_UNSUPPORTED
    assert lib.cosma_gemm(4, 4, emax, 16, emax, 16, 4, 16, 4, dt) == lib.COSMA_ERR_INVALID_ARG


def test_complex_k_limits_are_refused_before_any_staging(lib):
    # the complex entries reach the same limits as the real ones (their four real
    # products run on the same engines); the refusal precedes the pointer checks,
    # so it also precedes the sizing and allocation of the planar staging buffer
    cosma = lib
    al = 1.0 + 0j
    kmax, emax = 65535 * 32, 1023 * 2048
    assert cosma.cosma_cgemm(0, 0, 4, 4, kmax + 1, al, 0, kmax + 1, 0, 4, al, 0, 4,
                             cosma.COSMA_F32_EMU_TF32, 0) == cosma.COSMA_ERR_UNSUPPORTED
    assert cosma.cosma_zgemm(0, 0, 4, 4, emax + 1, al, 0, emax + 1, 0, 4, al, 0, 4,
                             cosma.COSMA_F64_EMU_BF16, 0) == cosma.COSMA_ERR_UNSUPPORTED
    # one element shorter: the same call fails on its null pointers instead
    assert cosma.cosma_cgemm(0, 0, 4, 4, kmax, al, 0, kmax, 0, 4, al, 0, 4,
                             cosma.COSMA_F32_EMU_TF32, 0) == cosma.COSMA_ERR_INVALID_ARG
    assert cosma.cosma_zgemm(0, 0, 4, 4, emax, al, 0, emax, 0, 4, al, 0, 4,
                             cosma.COSMA_F64_EMU_BF16, 0) == cosma.COSMA_ERR_INVALID_ARG
    # the engines without such a limit take the long k to the pointer checks
    assert cosma.cosma_cgemm(0, 0, 4, 4, kmax + 1, al, 0, kmax + 1, 0, 4, al, 0, 4,
                             cosma.COSMA_F32, 0) == cosma.COSMA_ERR_INVALID_ARG


def test_profile_host_rejects_bad_arguments(lib):
    import ctypes
    raw = lib.load()
    buf = (ctypes.c_double * 6)()
    assert raw.cosma_profile_host(None, 6) == lib.COSMA_ERR_INVALID_ARG
    assert raw.cosma_profile_host(buf, 0) == lib.COSMA_ERR_INVALID_ARG
    # without a device (or before any profiled host call) nothing is reported
    assert raw.cosma_profile_host(buf, 6) < 0


def test_host_entry_rejects_bad_arguments(lib):
    bad = lib.COSMA_ERR_INVALID_ARG
    assert lib.cosma_gemm_host(-1, 4, 4, 0, 4, 0, 4, 0, 4, lib.COSMA_F64) == bad
    assert lib.cosma_gemm_host(4, 4, 4, 0, 3, 0, 4, 0, 4, lib.COSMA_F64) == bad   # lda < k
    assert lib.cosma_gemm_host(4, 4, 4, 0, 4, 0, 4, 0, 2, lib.COSMA_F64) == bad   # ldc < n
    assert lib.cosma_gemm_host(4, 4, 4, 0, 4, 0, 4, 0, 4, lib.COSMA_F64) == bad   # null C
    assert lib.cosma_gemm_host(4, 4, 4, 8, 4, 8, 4, 8, 4, 9) == bad                 # dtype
    assert lib.cosma_gemm_host(0, 4, 4, 0, 4, 0, 4, 0, 4, lib.COSMA_F64) == lib.COSMA_OK


def test_init_validates_config(lib):
    assert lib.cosma_init(delta=1.5) == lib.COSMA_ERR_INVALID_ARG
    assert lib.cosma_init(selector=7) == lib.COSMA_ERR_INVALID_ARG
    assert lib.cosma_init(emu_slice_bits=9) == lib.COSMA_ERR_INVALID_ARG


@pytest.mark.parametrize("S", [3, 5, 10, 16, 37, 64, 100, 257, 1000, 4096, 61952, 247808])
def test_find_seq_schedule_matches_oracle(lib, S):
    assert lib.cosma_find_seq_schedule(S) == bounds.find_seq_schedule(S)


def test_fit_ranks_matches_oracle_random(lib):
    rng = random.Random(1234)
    for _ in range(150):
        m, n, k = (rng.randint(1, 3000) for _ in range(3))
        p = rng.randint(1, 90)
        delta = rng.choice([0.0, 0.03, 0.1, 0.25])
        assert lib.cosma_fit_ranks(m, n, k, p, delta) == bounds.fit_ranks(m, n, k, p, delta), \
            (m, n, k, p, delta)


def test_fit_ranks_paper_cases(lib):
    n = 4160
    assert lib.cosma_fit_ranks(n, n, n, 65, 0.03) == (4, 4, 4)                 # Fig. 6
    g1 = lib.cosma_fit_ranks(16384, 16384, 16384, 9216, 0.03)
    g2 = lib.cosma_fit_ranks(16384, 16384, 16384, 9217, 0.03)
    assert g1 == g2 == bounds.fit_ranks(16384, 16384, 16384, 9216, 0.03)       # Sec. 9


def _small_plan(lib, tile, kb, pk, order, ctas, pm=1, pn=1):
    p = lib.cosma_plan()
    p.kernel, p.tile_m, p.tile_n, p.k_block, p.stages = 0, tile[0], tile[1], kb, 2
    p.pm, p.pn, p.pk, p.order, p.ctas = pm, pn, pk, order, ctas
    return p


@pytest.mark.parametrize("order,pk,grid", [(1, 1, None), (1, 2, None), (0, 1, (2, 2)),
                                           (0, 2, (2, 1)), (1, 3, None)])
def test_plan_units_cover_iteration_space_once(lib, order, pk, grid):
    m, n, k = 11, 13, 9
    pm, pn = grid if grid else (1, 1)
    ctas = pm * pn * pk if order == 0 else 5
    p = _small_plan(lib, (4, 4), 2, pk, order, ctas, pm, pn)
    units = lib.cosma_plan_units(m, n, k, p)
    seen = {}
    for (r0, r1, c0, c1, k0, k1) in units:
        for i in range(r0, r1):
            for j in range(c0, c1):
                for t in range(k0, k1):
                    seen[(i, j, t)] = seen.get((i, j, t), 0) + 1
    assert len(seen) == m * n * k and set(seen.values()) == {1}


@pytest.mark.parametrize("order,pk", [(1, 1), (0, 1), (1, 2)])
def test_plan_replay_in_pebble_game(lib, order, pk):
    m, n, k = 16, 12, 10
    a, b = 4, 4
    pm, pn = (2, 3) if order == 0 else (1, 1)
    ctas = pm * pn * pk if order == 0 else 6
    p = _small_plan(lib, (a, b), 2, pk, order, ctas, pm, pn)
    units = lib.cosma_plan_units(m, n, k, p)
    # units of one k column must be replayed in k order for the partial-sum chain
    units = sorted(units, key=lambda u: (u[0], u[2], u[4]))
    S = pebble.listing1_working_set(a, b, sliding=False)
    res = pebble.simulate(m, n, k, S, pebble.plan_schedule(m, n, k, units), sliding=False)
    thm1 = bounds.thm1(m, n, k, S)
    assert res.io >= thm1
    if pk == 1:
        assert res.io == pebble.tile_io(m, n, k, a, b)
        assert res.io <= 1.3 * thm1


def test_plan_query_host_only(lib):
    # planning needs no GPU; every plan fits the kernel's limits
    for dt in (lib.COSMA_F64, lib.COSMA_F32):
        for shape in [(512, 512, 512), (16384, 16384, 16384), (4096, 4096, 1 << 20),
                      (1 << 20, 4096, 4096), (65536, 65536, 1024), (7, 129, 1000)]:
            p = lib.cosma_plan_query(*shape, dt)
            assert p.ctas >= 1 and p.pk >= 1
            assert p.io_words >= p.bound_words * 0.999 or shape[2] < 64
            if p.order == 0:
                assert p.pm * p.pn * p.pk == p.ctas
            sms = p.sms
            assert p.ctas <= sms
            assert p.ctas >= sms - math.floor(0.03 * sms) or p.ctas == p.pm * p.pn * p.pk \
                or p.ctas < sms


def test_plan_query_tf32_and_fp32_tiles_host_only(lib):
    # three-TF32 plans: the kernel's one 128 x 128 tile, 32-deep k blocks; the FMA
    # FP32 family takes its 128 x 256 tile where many tiles fill the waves and the
    # 128 x 128 one for small products
    for shape in [(16384, 16384, 16384), (4096, 4096, 4096), (300, 260, 515), (7, 129, 1000)]:
        p = lib.cosma_plan_query(*shape, lib.COSMA_F32_EMU_TF32)
        assert lib.KERNELS[p.kernel] == "tf32x3"
        assert (p.tile_m, p.tile_n, p.k_block) == (128, 128, 32)
        assert 1 <= p.ctas <= p.sms and 1 <= p.pk
    wide = lib.cosma_plan_query(16384, 16384, 16384, lib.COSMA_F32)
    assert (wide.tile_m, wide.tile_n) == (128, 256)
    small = lib.cosma_plan_query(512, 512, 512, lib.COSMA_F32)
    assert (small.tile_m, small.tile_n) == (128, 128)
    # the learned selector's candidate space does not include this dtype
    with pytest.raises(lib.CosmaError) as e:
        lib.cosma_plan_candidate(4096, 4096, 4096, lib.COSMA_F32_EMU_TF32, 0)
    assert e.value.status == lib.COSMA_ERR_INVALID_ARG


def test_plan_io_accounting_matches_units(lib):
    m, n, k = 512, 512, 512
    p = lib.cosma_plan_query(m, n, k, lib.COSMA_F64)
    units = lib.cosma_plan_units(m, n, k, p)
    io = 0
    for (r0, r1, c0, c1, k0, k1) in units:
        io += (k1 - k0) * ((r1 - r0) + (c1 - c0))
    io += m * n * (2 * p.pk + 1 if p.pk > 1 else 1)
    assert io == pytest.approx(p.io_words)


def test_plan_candidates_host_only(lib):
    for dt in (lib.COSMA_F64, lib.COSMA_F32, lib.COSMA_BF16, lib.COSMA_F64_EMU_BF16):
        for shape in [(4096, 4096, 4096), (300, 260, 70), (65536, 256, 1 << 16)]:
            valid = [c for c in range(lib.COSMA_MLP_OUT)
                     if lib.cosma_plan_candidate(*shape, dt, c) is not None]
            assert valid, (dt, shape)
            for c in valid:
                p = lib.cosma_plan_candidate(*shape, dt, c)
                assert p.pk == [1, 2, 4, 8][(c // 2) % 4] and p.order == c % 2
                assert 1 <= p.ctas <= p.sms
                if p.kernel == 3 and p.tile_m == 256:
                    assert p.ctas <= p.sms // 2
                if p.order == 0:
                    assert p.pm * p.pn * p.pk == p.ctas
            if dt == lib.COSMA_F64_EMU_BF16:
                assert valid == [1, 9]  # CTA-pair tile 256 x 256 and single-SM tile 128 x 128


def test_emu_plans_split_k_only_where_the_last_wave_is_short(lib):
    # largeK: 256 pair tiles over 76 SM pairs fill 3.4 of 4 rounds; a k split of
    # whole 4096-deep super-chunks evens the rounds out.  Square 16384^3 (4096
    # tiles, 54 rounds at 99.8 %) and flat k = 1024 (one super-chunk) stay unsplit.
    dt = lib.COSMA_F64_EMU_BF16
    p = lib.cosma_plan_query(4096, 4096, 1 << 20, dt)
    assert p.order == 1 and 1 < p.pk <= 16 and (p.tile_m, p.tile_n) == (256, 256)
    units = 16 * 16 * p.pk
    pairs = p.ctas
    assert units / (pairs * -(-units // pairs)) > 0.95  # the last round nearly full
    assert p.workspace_bytes >= 4096 * 4096 * 8        # the summed exact totals
    assert lib.cosma_plan_query(16384, 16384, 16384, dt).pk == 1
    assert lib.cosma_plan_query(65536, 65536, 1024, dt).pk == 1


@pytest.mark.parametrize("tile,pk", [((256, 256), 3), ((128, 128), 4), ((256, 128), 2)])
def test_emu_split_units_are_whole_super_chunks(lib, tile, pk):
    # k = 4 super-chunks and a ragged 100: every (tile, k slice) once, k slices
    # cut at multiples of 4096 and together covering [0, k); a CTA's units run
    # k slice first (slice number non-decreasing), so concurrent CTAs share one
    # k range
    m, n, k = 600, 520, 4 * 4096 + 100
    p = _small_plan(lib, tile, 64, pk, 1, 3)
    p.kernel = 3
    units = lib.cosma_plan_units(m, n, k, p)
    tiles = -(-m // tile[0]) * -(-n // tile[1])
    assert len(units) == tiles * pk
    per_tile = {}
    for (r0, r1, c0, c1, k0, k1) in units:
        assert k0 % 4096 == 0 and (k1 % 4096 == 0 or k1 == k) and k0 < k1
        per_tile.setdefault((r0, c0), []).append((k0, k1))
    assert len(per_tile) == tiles
    for ranges in per_tile.values():
        ranges.sort()
        assert ranges[0][0] == 0 and ranges[-1][1] == k
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    # units come back CTA by CTA; inside a CTA the k slice never goes back
    pos = 0
    for c in range(3):
        count = len(range(c, tiles * pk, 3))
        starts = [u[4] for u in units[pos:pos + count]]
        assert starts == sorted(starts)
        pos += count


def test_selector_features_match_oracle(lib):
    from oracle import mlp as om
    import numpy as np
    for (m, n, k, dt) in [(256, 65536, 1024, 2), (3, 5, 7, 0), (4096, 1, 2, 3)]:
        got = np.array(lib.cosma_selector_features(m, n, k, dt))
        assert np.allclose(got, om.features(m, n, k, dt), rtol=1e-6, atol=1e-7)


def test_gemm_ex_rejects_short_leading_dimensions(lib):
    cosma = lib
    # trans_a: A is k x m, so lda >= m; trans_b: B is n x k, so ldb >= k
    assert cosma.cosma_gemm_ex(1, 0, 8, 4, 16, 1.0, 1, 7, 1, 4, 0.0, 1, 4,
                               cosma.COSMA_F64, 0) == cosma.COSMA_ERR_INVALID_ARG
    assert cosma.cosma_gemm_ex(0, 1, 8, 4, 16, 1.0, 1, 16, 1, 15, 0.0, 1, 4,
                               cosma.COSMA_F64, 0) == cosma.COSMA_ERR_INVALID_ARG
    assert cosma.cosma_gemm_ex(2, 0, 8, 4, 16, 1.0, 1, 16, 1, 4, 0.0, 1, 4,
                               cosma.COSMA_F64, 0) == cosma.COSMA_ERR_INVALID_ARG


def test_zgemm_rejects_other_engines_and_bad_ops(lib):
    cosma = lib
    al = 1.0 + 0j
    assert cosma.cosma_zgemm(0, 0, 4, 4, 4, al, 0, 4, 0, 4, al, 0, 4,
                             cosma.COSMA_BF16, 0) == cosma.COSMA_ERR_UNSUPPORTED
    assert cosma.cosma_zgemm(3, 0, 4, 4, 4, al, 0, 4, 0, 4, al, 0, 4,
                             cosma.COSMA_F64, 0) == cosma.COSMA_ERR_INVALID_ARG
    assert cosma.cosma_zgemm(1, 0, 8, 4, 4, al, 0, 7, 0, 4, al, 0, 4,
                             cosma.COSMA_F64, 0) == cosma.COSMA_ERR_INVALID_ARG  # lda < m


def test_cgemm_rejects_other_engines_and_bad_arguments(lib):
    cosma = lib
    al = 1.0 + 0j
    for eng in (cosma.COSMA_F64, cosma.COSMA_BF16, cosma.COSMA_F64_EMU_BF16):
        assert cosma.cosma_cgemm(0, 0, 4, 4, 4, al, 0, 4, 0, 4, al, 0, 4,
                                 eng, 0) == cosma.COSMA_ERR_UNSUPPORTED
    assert cosma.cosma_cgemm(0, 3, 4, 4, 4, al, 0, 4, 0, 4, al, 0, 4,
                             cosma.COSMA_F32, 0) == cosma.COSMA_ERR_INVALID_ARG
    assert cosma.cosma_cgemm(0, 2, 4, 8, 6, al, 0, 6, 0, 5, al, 0, 8,
                             cosma.COSMA_F32_EMU_TF32, 0) == cosma.COSMA_ERR_INVALID_ARG  # ldb < k
    assert cosma.cosma_cgemm(0, 0, 0, 4, 4, al, 0, 4, 0, 4, al, 0, 4,
                             cosma.COSMA_F32, 0) == cosma.COSMA_OK  # m == 0: nothing to do



def test_environment_sets_config_defaults(lib):
    """COSMA_* variables are read when the library loads (a fresh process here);
    bad values leave the built-in default."""
    import json
    import subprocess
    import sys
    code = ("from paper_1908_09606_gb300 import cosma; cosma.load(); c = cosma.cosma_get_config(); "
            "import json; print(json.dumps([c.delta, c.selector, c.emu_slices, "
            "c.emu_slice_bits, c.wait_limit, c.grouped_tile]))")
    env = dict(os.environ, COSMA_DELTA="0.1", COSMA_SELECTOR="learned", COSMA_EMU_SLICES="7",
               COSMA_EMU_SLICE_BITS="7", COSMA_WAIT_LIMIT="12345", COSMA_GROUPED_TILE="256")
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True,
                         text=True, check=True).stdout
    assert json.loads(out) == [0.1, 1, 7, 7, 12345, 256]
    env = dict(os.environ, COSMA_DELTA="1.5", COSMA_SELECTOR="fast", COSMA_EMU_SLICES="x",
               COSMA_GROUPED_TILE="100")
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True,
                         text=True, check=True).stdout
    assert json.loads(out) == [0.03, 0, 0, 0, 0, 0]


def test_planner_units_partition_random_shapes(lib):
    """Property: for any shape and dtype the planner's own plan has units that
    partition the iteration space -- tiles cover C once, and each tile's k
    ranges partition [0, k) -- and fits the grid it claims."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=60, deadline=None, derandomize=True)
    @hyp.given(m=st.integers(1, 3000), n=st.integers(1, 3000), k=st.integers(1, 40000),
               dt=st.sampled_from([0, 1, 2, 3, 5]))
    def check(m, n, k, dt):
        p = lib.cosma_plan_query(m, n, k, dt)
        assert 1 <= p.ctas <= p.sms and p.pk >= 1
        units = lib.cosma_plan_units(m, n, k, p)
        tiles = {}
        for (r0, r1, c0, c1, k0, k1) in units:
            assert 0 <= r0 < r1 <= m and 0 <= c0 < c1 <= n and 0 <= k0 < k1 <= k
            assert r0 % p.tile_m == 0 and c0 % p.tile_n == 0
            assert r1 == min(r0 + p.tile_m, m) and c1 == min(c0 + p.tile_n, n)
            tiles.setdefault((r0, c0), []).append((k0, k1))
        assert len(tiles) == -(-m // p.tile_m) * -(-n // p.tile_n)
        for ranges in tiles.values():
            ranges.sort()
            assert ranges[0][0] == 0 and ranges[-1][1] == k and len(ranges) == p.pk
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))

    check()
