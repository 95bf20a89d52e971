"""The batched small-state engine: host compilation (CPU) and GPU parity of
many independent circuits run in one persistent launch against the oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2308_01999_gb300 import inputs as gen


@pytest.fixture(scope="module")
def svmod():
    from paper_2308_01999_gb300 import _build
    _build.build()
    from paper_2308_01999_gb300 import sv
    sv.lib()
    return sv


def _mixed_states(seed, sizes, strings=5):
    rng = gen.rng_for(seed)
    states = []
    x = np.array([[0, 1], [1, 0]], dtype=complex)
    y = np.array([[0, -1j], [1j, 0]])
    for i, n in enumerate(sizes):
        if i % 4 == 0:
            gates = gen.ansatz_circuit(n, 3, rng)
        elif i % 4 == 1:
            gates = gen.layered_random_circuit(n, 3, seed + i, ("cz", "cnot", "crz")) if n >= 2 else \
                [gen.Gate((0,), gen.haar_su2(rng))]
        elif i % 4 == 3 and n >= 3:
            # permutations on a few qubits, so that they share register windows:
            # X, X controlled on 0 or 1, Toffoli-like with random control values,
            # controlled Y (factors +-i), and Haar gates in between
            pool = [int(v) for v in rng.choice(n, min(n, 5), replace=False)]
            gates = []
            for _ in range(24):
                qs = [int(v) for v in rng.choice(pool, 3, replace=False)]
                kind = int(rng.integers(0, 5))
                cv = tuple(int(v) for v in rng.integers(0, 2, size=2))
                if kind == 0:
                    gates.append(gen.Gate((qs[0],), gen.haar_su2(rng)))
                elif kind == 1:
                    gates.append(gen.Gate((qs[0],), x))
                elif kind == 2:
                    gates.append(gen.Gate((qs[0],), x, (qs[1],), cv[:1]))
                elif kind == 3:
                    gates.append(gen.Gate((qs[0],), x, (qs[1], qs[2]), cv))
                else:
                    gates.append(gen.Gate((qs[0],), y, (qs[1],), cv[:1]))
        else:
            gates = []
            for _ in range(12):
                k = int(rng.integers(1, min(3, n) + 1))
                c = int(rng.integers(0, min(2, n - k) + 1))
                qs = [int(x) for x in rng.choice(n, k + c, replace=False)]
                gates.append(gen.Gate(tuple(qs[:k]), gen.random_gate_dense(rng, k), tuple(qs[k:]),
                                      tuple(int(v) for v in rng.integers(0, 2, size=c))))
        paulis, _ = gen.random_pauli_strings(n, strings, rng)
        states.append((n, gates, paulis))
    return states


def test_compile_on_host_only(svmod):
    sv = svmod
    b = sv.Batch()
    states = _mixed_states(1, [3, 10, 14, 16, 18])
    info = b.compile(states, fusion_width=2)
    assert info["items"] == 5 and info["launches"] == 0
    assert info["state_amps"] == sum(1 << n for n, _, _ in states)
    # states of <= 14 qubits take one pass; larger ones need more than one
    one = sv.Batch()
    assert one.compile(states[:3], 3)["stages"] == 3
    assert info["stages"] > 5
    # runs of small ops on at most 4 qubits become register windows: a 14-qubit
    # ansatz compiled without fusion needs far fewer ops than it has gates
    rng = gen.rng_for(5)
    ans = gen.ansatz_circuit(14, 3, rng)
    w = sv.Batch()
    assert w.compile([(14, ans, np.zeros((0, 14)))], 1)["ops"] < len(ans) / 3
    # the window width is an option: no windows leave one op per (fused) gate
    plain = w.compile([(14, ans, np.zeros((0, 14)))], 1, window_qubits=0)["ops"]
    assert plain > 2 * w.compile([(14, ans, np.zeros((0, 14)))], 1, window_qubits=3)["ops"]
    for bad in (1, 5, -1):
        with pytest.raises(sv.SvError):
            w.compile([(14, ans, np.zeros((0, 14)))], 1, window_qubits=bad)
    w.close()
    with pytest.raises(sv.SvError):
        sv.Batch().compile([(3, [gen.Gate((3,), np.eye(2))], np.zeros((0, 3)))], 2)
    with pytest.raises(sv.SvError):
        sv.Batch().compile([(27, [], np.zeros((0, 27)))], 2)      # above SV_BATCH_MAX_QUBITS
    with pytest.raises(sv.SvError):
        sv.Batch().compile(states, 5)
    b.close()


def test_tile_size_option_on_host(svmod):
    """tile_qubits sets the local qubits of a pass: a state at or below it is
    one pass, a state above it several; a tile of 12 takes register windows of
    at most 3 qubits (2^(T - w) groups must cover the CTA), so the same
    program needs more ops; a gate wider than the tile is rejected, and so is
    a tile outside 10..14."""
    import ctypes as C
    sv = svmod
    rng = gen.rng_for(9)
    big = (16, gen.ansatz_circuit(16, 3, rng), np.zeros((0, 16)))
    small = (12, gen.ansatz_circuit(12, 3, rng), np.zeros((0, 12)))
    ops = {}
    for tile in (14, 13, 12):
        b = sv.Batch()
        info = b.compile([big], 2, 4, False, tile)
        assert b.choice == (2, 4, 0, tile) and info["stages"] >= 2
        ops[tile] = info["ops"]
        assert b.compile([small], 2, 4, False, tile)["stages"] == 1
        b.close()
    assert ops[12] > ops[14]
    wide = (13, [gen.Gate((0, 1, 2, 3), gen.random_gate_dense(rng, 4), tuple(range(4, 13)), (1,) * 9)],
            np.zeros((0, 13)))
    b = sv.Batch()
    with pytest.raises(sv.SvError):
        b.compile([wide], 2, 4, False, 12)           # 13 qubits on one gate, tile of 12
    b.close()
    packed = sv.pack_batch([small])
    h = C.c_void_p()
    assert sv.lib().sv_batch_create(None, C.byref(h)) == 0
    try:
        for bad in (9, 15, 0):
            opt = (C.c_int * 4)(2, 4, 0, bad)
            rc = sv.lib().sv_batch_compile_ex(h, C.c_void_p(packed.items.ctypes.data), len(packed.items),
                                              C.c_void_p(packed.gate_rec.ctypes.data), len(packed.gate_rec),
                                              None, C.cast(opt, C.c_void_p))
            assert rc == 1, (bad, rc)                  # SV_ERR_INVALID_ARGUMENT
    finally:
        sv.lib().sv_batch_destroy(h)


def test_keep_permutations_rule_on_host(svmod):
    """With keep_permutations, a fused block that starts with a CNOT, X or
    other permutation takes no dense gate: CNOTs on disjoint pairs, each
    followed by Haar gates on both of its qubits, fuse to one dense block per
    pair without the rule and to a permutation block plus a dense block per
    pair with it; an option value other than 0 or 1 is rejected."""
    import ctypes as C
    sv = svmod
    rng = gen.rng_for(8)
    x = np.array([[0, 1], [1, 0]], dtype=complex)
    n = 12
    gates = []
    for _ in range(4):
        gates += [gen.Gate((q + 1,), x, (q,), (1,)) for q in range(0, n, 2)]
        gates += [gen.Gate((q,), gen.haar_su2(rng)) for q in range(n)]
    prog = [(n, gates, np.zeros((0, n)))]
    ops = {}
    for keep in (False, True):
        b = sv.Batch()
        ops[keep] = b.compile(prog, 2, 0, keep)["ops"]
        assert b.choice == (2, 0, int(keep), 14)
        b.close()
    assert ops[False] == n // 2 and ops[True] == n
    packed = sv.pack_batch(prog)
    h = C.c_void_p()
    assert sv.lib().sv_batch_create(None, C.byref(h)) == 0
    try:
        for bad in ((2, 4, 2), (2, 4, -1)):
            opt = (C.c_int * 4)(*bad, 14)
            rc = sv.lib().sv_batch_compile_ex(h, C.c_void_p(packed.items.ctypes.data), len(packed.items),
                                              C.c_void_p(packed.gate_rec.ctypes.data), len(packed.gate_rec),
                                              None, C.cast(opt, C.c_void_p))
            assert rc == 1, (bad, rc)                  # SV_ERR_INVALID_ARGUMENT
    finally:
        sv.lib().sv_batch_destroy(h)


@pytest.mark.gpu
@pytest.mark.parametrize("width,window,keep,tile", [(1, 4, 0, 14), (2, 4, 0, 14), (3, 4, 0, 14), (4, 4, 0, 14),
                                                    (1, 0, 0, 14), (2, 2, 0, 14), (1, 3, 0, 14), (2, 4, 1, 14),
                                                    (3, 4, 1, 14), (2, 3, 1, 14), (4, 0, 1, 14), (2, 4, 0, 13),
                                                    (2, 3, 0, 12), (3, 4, 0, 10)])
def test_batch_matches_oracle(svmod, width, window, keep, tile):
    import torch
    sv = svmod
    # every fourth state (i % 4 == 3) is the permutation mix; the 15- and
    # 13-qubit ones run it through 4-qubit register windows
    sizes = [1, 2, 5, 10, 12, 13, 14, 15, 16, 17, 18, 4, 11, 14, 16, 13, 12, 20]
    states = _mixed_states(10 + width, sizes)
    b = sv.Batch(torch.cuda.current_stream())
    b.compile(states, fusion_width=width, window_qubits=window, keep_permutations=bool(keep), tile_qubits=tile)
    buf = torch.zeros(b.state_amps, dtype=torch.complex64, device="cuda")
    b.launch(buf, keep_states=True)
    res = b.results()
    host = buf.cpu().numpy()
    for (n, gates, paulis), (off, _, _, _), got in zip(states, b.offsets, res):
        ref = orc.run_circuit(gates, n)
        amp = host[off:off + (1 << n)].astype(np.complex128)
        err = np.max(np.abs(amp - ref))
        assert err <= 1e-5, (n, width, err)
        want = np.array([orc.expect_pauli(ref, p, list(range(n))).real for p in paulis])
        assert np.all(np.abs(got - want) <= 1e-6 * np.maximum(1, np.abs(want))), (n, got, want)
    b.close()


@pytest.mark.gpu
def test_batch_equals_single_state_path_and_repeats(svmod):
    """The same circuits through sv_apply_matrix + sv_expectation_pauli one
    state at a time; a second launch of the same program gives the same values."""
    import torch
    sv = svmod
    states = _mixed_states(77, [10, 12, 14, 16, 20], strings=8)
    b = sv.Batch(torch.cuda.current_stream())
    b.compile(states, fusion_width=2)
    buf = torch.zeros(b.state_amps, dtype=torch.complex64, device="cuda")
    b.launch(buf)
    first = [r.copy() for r in b.results()]
    b.launch(buf)
    second = b.results()
    for a, c in zip(first, second):
        assert np.array_equal(a, c)
    for (n, gates, paulis), got in zip(states, first):
        psi = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
        s = sv.StateVector(psi)
        s.set_basis_state(0)
        s.apply_circuit(gates)
        want = s.expectation_pauli(paulis, np.tile(np.arange(n, dtype=np.int32), (paulis.shape[0], 1)))
        assert np.all(np.abs(got - want) <= 1e-6 * np.maximum(1, np.abs(want))), (n, got, want)
        s.close()
    b.close()


@pytest.mark.gpu
def test_gate_launches_replay_from_a_cuda_graph(svmod):
    """The per-gate launches of sv_apply_matrix can be captured in a CUDA graph
    (no allocation, synchronisation or pageable copy on that path for gates of
    up to 4 targets) and replayed; the replay reproduces the direct run bit for
    bit."""
    import torch
    sv = svmod
    n = 12
    states = _mixed_states(31, [n, n, n])
    stream = torch.cuda.Stream()
    for _, gates, _ in states:
        direct = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
        d = sv.StateVector(direct, stream)
        with torch.cuda.stream(stream):
            d.set_basis_state(0)
            d.apply_circuit(gates)
        stream.synchronize()
        psi = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
        s = sv.StateVector(psi, stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            s.set_basis_state(0)
            s.apply_circuit(gates)
        psi.fill_(0)
        torch.cuda.synchronize()
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(psi, direct)
        s.close()
        d.close()


@pytest.mark.gpu
def test_empty_programs(svmod):
    """A batch of no states launches nothing (an empty state buffer is
    accepted); states without gates stay |0...0>, in shared memory (12 qubits)
    and tiled through global memory (16 qubits): <Z...Z> = <I> = 1 and any
    string with an X or a Y gives 0."""
    import torch
    sv = svmod
    b = sv.Batch(torch.cuda.current_stream())
    info = b.compile([], 2)
    assert info["items"] == 0 and info["state_amps"] == 0
    b.launch(torch.empty(0, dtype=torch.complex64, device="cuda"))
    assert b.results() == []
    states = []
    for n in (12, 16):
        p = np.zeros((4, n), np.int32)
        p[0, :] = 3
        p[2, 0] = 1
        p[3, :2] = [2, 3]
        states.append((n, [], p))
    b.compile(states, 2)
    buf = torch.zeros(b.state_amps, dtype=torch.complex64, device="cuda")
    b.launch(buf)
    for got in b.results():
        assert np.allclose(got, [1.0, 1.0, 0.0, 0.0], atol=1e-12), got
    b.close()


@pytest.mark.gpu
@pytest.mark.parametrize("window", [4, 0])
def test_register_window_exchange_cases(svmod, window):
    """CNOTs folded into the one-qubit product before them, inside one 4-qubit
    register window of a 13-qubit state: the product on the exchange's target
    and on its control, control values 1 and 0, and a product that moves
    forward past an op on other qubits; with windows off the same circuit runs
    op by op. Amplitudes against the oracle."""
    import torch
    sv = svmod
    n = 13
    rng = gen.rng_for(404)
    x = np.array([[0, 1], [1, 0]], dtype=complex)
    g = [gen.Gate((q,), gen.haar_su2(rng)) for q in range(n)]
    g += [gen.Gate((0,), gen.haar_su2(rng)), gen.cnot(0, 1),                  # product on the control
          gen.Gate((2,), gen.haar_su2(rng)), gen.Gate((3,), x, (2,), (0,)),   # control value 0
          gen.Gate((1,), gen.haar_su2(rng)), gen.Gate((3,), gen.haar_su2(rng)),
          gen.cnot(0, 1),                                                     # product on the target,
          gen.cnot(3, 2),                                                     # past the op on qubit 3
          gen.Gate((0,), gen.haar_su2(rng)), gen.Gate((0,), x, (1,), (0,)),   # target, control value 0
          gen.Gate((2,), gen.haar_su2(rng)), gen.cz(1, 2), gen.cnot(2, 3)]
    paulis, _ = gen.random_pauli_strings(n, 4, rng)
    b = sv.Batch(torch.cuda.current_stream())
    b.compile([(n, g, paulis)], fusion_width=1, window_qubits=window)
    buf = torch.zeros(b.state_amps, dtype=torch.complex64, device="cuda")
    b.launch(buf, keep_states=True)
    res = b.results()[0]
    ref = orc.run_circuit(g, n)
    amp = buf.cpu().numpy()[:1 << n].astype(np.complex128)
    assert np.max(np.abs(amp - ref)) <= 1e-5
    want = np.array([orc.expect_pauli(ref, p, list(range(n))).real for p in paulis])
    assert np.all(np.abs(res - want) <= 1e-6 * np.maximum(1, np.abs(want)))
    b.close()


@pytest.mark.gpu
@pytest.mark.parametrize("window", [4, 3, 0])
def test_register_window_exchange_first_cases(svmod, window):
    """CNOTs fused with the one-qubit product after them (the product moves
    back to the exchange and reads the exchanged registers), where a CZ on the
    same qubits stops a fold with the product before them: the product on the
    exchange's target and on its control, control values 1 and 0, and a
    product that moves back past an op on another qubit; windows of 4 and 3
    qubits and none. Amplitudes and expectations against the oracle."""
    import torch
    sv = svmod
    n = 13
    rng = gen.rng_for(405)
    x = np.array([[0, 1], [1, 0]], dtype=complex)
    h = lambda q: gen.Gate((q,), gen.haar_su2(rng))         # noqa: E731
    g = [h(q) for q in range(n)]
    g += [gen.cz(0, 1), gen.cnot(0, 1), h(1)]                      # product on the target, value 1
    g += [gen.cz(2, 3), gen.Gate((3,), x, (2,), (0,)), h(2)]       # product on the control, value 0
    g += [gen.cz(0, 3), gen.cnot(3, 0), h(1), h(3)]                # on the control, past an op on qubit 1
    g += [gen.cz(1, 2), gen.Gate((1,), x, (2,), (0,)), h(1)]       # on the target, value 0
    g += [gen.cz(0, 2), gen.cnot(2, 0), h(2)]                      # on the control, value 1
    g += [h(q) for q in range(4)]
    paulis, _ = gen.random_pauli_strings(n, 4, rng)
    for width in (1, 2):
        b = sv.Batch(torch.cuda.current_stream())
        b.compile([(n, g, paulis)], fusion_width=width, window_qubits=window)
        buf = torch.zeros(b.state_amps, dtype=torch.complex64, device="cuda")
        b.launch(buf, keep_states=True)
        res = b.results()[0]
        ref = orc.run_circuit(g, n)
        amp = buf.cpu().numpy()[:1 << n].astype(np.complex128)
        assert np.max(np.abs(amp - ref)) <= 1e-5, (width, window)
        want = np.array([orc.expect_pauli(ref, p, list(range(n))).real for p in paulis])
        assert np.all(np.abs(res - want) <= 1e-6 * np.maximum(1, np.abs(want))), (width, window)
        b.close()


def test_cnot_times_one_qubit_blocks_are_split_on_host(svmod):
    """A fused two-qubit block that is a CNOT times a one-qubit gate on one of
    its qubits (either order) is compiled as the 2x2 product fused with the
    exchange inside a register window, not as one 4x4 product; a block with
    one-qubit gates on both qubits stays a 4x4 product, and without windows
    nothing is split (each part would be a pass of its own)."""
    sv = svmod
    rng = gen.rng_for(406)
    n = 14
    h = lambda q: gen.Gate((q,), gen.haar_su2(rng))         # noqa: E731
    cases = {
        "gate then cnot, gate on control": [h(0), gen.cnot(0, 1)],
        "gate then cnot, gate on target": [h(1), gen.cnot(0, 1)],
        "cnot then gate on control": [gen.cnot(0, 1), h(0)],
        "cnot then gate on target, control value 0": [gen.Gate((1,), np.array([[0, 1], [1, 0]], complex), (0,), (0,)),
                                                       h(1)],
        "gates on both qubits": [h(0), h(1), gen.cnot(0, 1)],
    }
    for name, gates in cases.items():
        both = name == "gates on both qubits"
        b = sv.Batch()
        b.compile([(n, gates, np.zeros((0, n)))], 2, 4)
        st = b.program_stats()
        if both:          # one 4x4 product (a window of one op is emitted as the op)
            assert st["win_4x4"] + st["dense_ops"] == 1 and st["win_2x2"] == 0, (name, st)
        else:
            assert st["windows"] == 1 and st["dense_ops"] == 0 and st["win_4x4"] == 0, (name, st)
            assert st["win_2x2"] == st["win_2x2_with_exchange"] == 1, (name, st)
        assert b.compile([(n, gates, np.zeros((0, n)))], 2, 0)["ops"] == 1      # no windows: no split
        assert b.program_stats()["dense_ops"] == 1
        b.close()
    # before a compile, and with no output array, the stats call is rejected
    import ctypes as C
    h = C.c_void_p()
    assert sv.lib().sv_batch_create(None, C.byref(h)) == 0
    try:
        out = (C.c_uint64 * sv.SV_BATCH_STATS)()
        assert sv.lib().sv_batch_program_stats(h, out) == 1            # SV_ERR_INVALID_ARGUMENT
        assert sv.lib().sv_batch_program_stats(h, None) == 1
    finally:
        sv.lib().sv_batch_destroy(h)


@pytest.mark.gpu
def test_large_states_split_over_the_gpu_match_the_oracle(svmod):
    """States of 15-24 qubits: every pass of their circuits is split into tile
    tasks that many CTAs share, and their expectation sums into chunks; next to
    them, states that fit one CTA. Amplitudes and expectation values against the
    oracle, in several fusion and window settings."""
    import torch
    sv = svmod
    orc.set_threads(0)
    sizes = [21, 12, 15, 24, 16, 9, 22]
    states = _mixed_states(2024, sizes, strings=6)
    refs = [orc.run_circuit(g, n) for n, g, _ in states]
    for width, window, keep, tile in ((2, 4, 0, 14), (1, 0, 0, 14), (3, 3, 0, 14), (2, 4, 1, 14), (2, 3, 0, 12)):
        b = sv.Batch(torch.cuda.current_stream())
        b.compile(states, fusion_width=width, window_qubits=window, keep_permutations=bool(keep), tile_qubits=tile)
        buf = torch.zeros(b.state_amps, dtype=torch.complex64, device="cuda")
        b.launch(buf, keep_states=True)
        res = b.results()
        host = buf.cpu().numpy()
        for (n, gates, paulis), (off, _, _, _), got, ref in zip(states, b.offsets, res, refs):
            amp = host[off:off + (1 << n)].astype(np.complex128)
            err = np.max(np.abs(amp - ref))
            assert err <= 1e-5, (n, width, window, err)
            want = np.array([orc.expect_pauli(ref, p, list(range(n))).real for p in paulis])
            assert np.all(np.abs(got - want) <= 1e-6 * np.maximum(1, np.abs(want))), (n, got, want)
        b.close()


@pytest.mark.gpu
def test_results_do_not_depend_on_the_rest_of_the_batch(svmod):
    """A state's expectation values are bit for bit the same alone and inside a
    batch of other states, for states that fit one CTA and states split over
    many (per-chunk partial sums added in a fixed order)."""
    import torch
    sv = svmod
    mix = _mixed_states(99, [18, 11, 20, 14, 16, 13, 19], strings=5)
    b = sv.Batch(torch.cuda.current_stream())
    b.compile(mix, fusion_width=2)
    buf = torch.zeros(b.state_amps, dtype=torch.complex64, device="cuda")
    b.launch(buf)
    together = [r.copy() for r in b.results()]
    for i in (0, 1, 2, 3):
        b.compile([mix[i]], fusion_width=2)
        b.launch(buf)
        alone = b.results()[0]
        assert np.array_equal(alone, together[i]), i
    b.close()


@pytest.mark.gpu
def test_full_batched_workload_sampled_against_the_oracle(svmod):
    """The benchmark's whole batched workload (4096 states of 10-20 qubits,
    6-layer ansatz, 8 Pauli strings each) in the launch configuration the
    benchmark times (fusion width 2, windows of 4 qubits, every state on one
    CTA): a stratified sample of 24 states, one per size step, compared with
    the complex128 oracle one by one."""
    import torch
    from paper_2308_01999_gb300 import autotune
    sv = svmod
    orc.set_threads(0)
    work = gen.batched_ansatz_workload(count=4096, seed=3)
    states = [(n, g, p) for n, g, p, _ in work]
    b = sv.Batch(torch.cuda.current_stream())
    info = b.compile(states, fusion_width=2, window_qubits=4)
    assert info["items"] == 4096
    buf = torch.empty(b.state_amps, dtype=torch.complex64, device="cuda")
    b.launch(buf)
    res = b.results()
    idx = autotune.stratified_sample([n for n, _, _ in states], 24)
    worst = 0.0
    for i in idx:
        n, gates, paulis = states[i]
        ref = orc.run_circuit(gates, n)
        want = np.array([orc.expect_pauli(ref, p, list(range(n))).real for p in paulis])
        d = np.abs(res[i] - want)
        worst = max(worst, float(d.max()))
        assert np.all(d <= 1e-6 * np.maximum(1, np.abs(want))), (i, n, res[i], want)
    print(f"[batch 4096] {len(idx)} sampled states: max |d<P>| {worst:.3e}")
    b.close()
