"""Host-side checks of the fused-pass planner (no GPU): pass counts and the
algorithmic cost model (HBM bytes, floating-point operations) that the
roofline of a fused pass is measured against."""
import math
import os

import pytest

from paper_2508_15545_gb300.workloads import Gate, random_circuit, config_seed, layer_count_gates


@pytest.fixture(scope="module")
def qv(qvlib):
    return qvlib


def cost(qv, n, gates, dtype=0, **kw):
    return qv.qv_plan_cost(n, dtype, gates, **kw)


@pytest.mark.parametrize("dtype,ab", [(0, 8), (1, 16)])
def test_single_gate_cost(qv, dtype, ab):
    n, N = 12, 1 << 12
    u3 = Gate("u3", 0, theta=(0.3, 0.2, 0.1))
    c = cost(qv, n, [u3], dtype, tile_bits=10)
    assert c["bytes"] == 2 * N * ab          # one read + one write of the state
    assert c["flops"] == 14 * N              # Eq. 5: 28 real operations per pair
    info = qv.qv_plan_info(n, dtype, [u3], tile_bits=10)
    assert info["passes"] == 1 and info["ops"] == 1


def test_op_kinds_cost(qv):
    n, N = 12, 1 << 12
    assert cost(qv, n, [Gate("x", 3, ctrl=0)], tile_bits=10)["flops"] == 0          # CNOT: a permutation
    assert cost(qv, n, [Gate("z", 3, ctrl=0)], tile_bits=10)["flops"] == 0          # CZ: sign flips only
    assert cost(qv, n, [Gate("p", 3, ctrl=0, theta=(0.5, 0, 0))], tile_bits=10)["flops"] == 3 * N  # CP: diagonal, half
    assert cost(qv, n, [Gate("rz", 5, theta=(0.7, 0, 0))], tile_bits=10)["flops"] == 6 * N
    assert cost(qv, n, [Gate("u3", 4, ctrl=1, theta=(0.3, 0.2, 0.1))], tile_bits=10)["flops"] == 7 * N


def test_fusion_reduces_flops(qv):
    n, N = 12, 1 << 12
    gates = [Gate("h", 2), Gate("ry", 2, theta=(0.4, 0, 0)), Gate("h", 2)]
    fused = cost(qv, n, gates, tile_bits=10)
    unfused = cost(qv, n, gates, tile_bits=10, flags=qv.QV_PLAN_NO_FUSION)
    assert fused["flops"] == 14 * N
    assert unfused["flops"] == 3 * 14 * N
    assert fused["bytes"] == unfused["bytes"] == 2 * N * 8


def test_high_qubits_join_the_tile(qv):
    # gates on qubits far above the contiguous low run still share one pass
    n = 20
    gates = [Gate("h", q) for q in (19, 15, 11, 0)]
    info = qv.qv_plan_info(n, 0, gates, tile_bits=10)
    assert info["passes"] == 1


@pytest.mark.parametrize("k", [10, 11, 12])
def test_random_circuit_30q_cost_consistent(qv, k):
    n, layers = 30, 40
    gates = random_circuit(n, layers, config_seed(1))
    assert len(gates) == layer_count_gates(n, layers) == 1780
    info = qv.qv_plan_info(n, 0, gates, tile_bits=k)
    c = cost(qv, n, gates, tile_bits=k)
    N = 1 << n
    assert c["bytes"] == 2 * info["passes"] * N * 8
    # 1200 U3 (14 per amplitude) at most; fusion only removes work
    assert 0 < c["flops"] <= 1200 * 14 * N
    # every pass holds at least one gate; the tiles leave at most n - k qubits out
    assert 1 <= info["passes"] <= len(gates)
    assert info["ops"] <= len(gates)
    assert math.isfinite(c["flops"])


def test_plan_cost_rejects_bad_args(qv):
    with pytest.raises(qv.QvError):
        qv.qv_plan_cost(0, 0, [Gate("h", 0)])
    with pytest.raises(qv.QvError):
        qv.qv_plan_cost(12, 0, [Gate("h", 12)], tile_bits=10)


@pytest.mark.parametrize("flags", [0, 1, 2])
def test_swap_of_two_outside_qubits_first(qv, flags):
    """A SWAP of two qubits outside the low chunk heads the gate list and every
    other gate waits behind it (controlled by one of its qubits), while other
    qubits are wanted as targets more often: the tile must still take both
    qubits of the SWAP, or the planner makes no progress."""
    n = 15
    gates = [Gate("swap", 10, target2=8)]
    for q in (5, 6, 7, 9, 11, 12, 13, 14):
        gates += [Gate("x", q, ctrl=10)] * 10
    info = qv.qv_plan_info(n, 0, gates, tile_bits=10, flags=flags)
    assert info["passes"] >= 1



def _compile_or_skip(qv, *args, **kw):
    try:
        return qv.qv_plan_compile(*args, **kw)
    except qv.QvError as e:
        if e.status == qv.QV_ERR_UNSUPPORTED:
            pytest.skip(f"NVRTC unavailable: {e}")
        raise


# (dtype, tile bits, flags): compiled engine with fusion and pair ops, no
# fusion, fusion without pair ops; complex128
@pytest.mark.parametrize("dtype,k,flags", [(0, 10, 0), (0, 11, 0), (0, 12, 0), (0, 11, 1), (0, 12, 4),
                                           (1, 10, 0), (1, 12, 0)])
def test_generated_passes_compile_on_host(qv, dtype, k, flags):
    """Every pass kernel the compiled engine would generate for a circuit of
    every gate kind (controls inside and outside the tile, SWAPs) compiles with
    NVRTC for sm_103a, without a GPU."""
    from paper_2508_15545_gb300 import workloads as W
    n = 13
    gates = W.random_gate_list(n, 160, seed=700 + 10 * k + dtype, ctrl_prob=0.4)
    info = qv.qv_plan_info(n, dtype, gates, tile_bits=k, flags=flags)
    got = _compile_or_skip(qv, n, dtype, gates, tile_bits=k, flags=flags)
    assert got["passes"] == info["passes"] and got["source_bytes"] > 0


def test_bench_like_circuit_compiles_on_host(qv):
    """The passes of a 20-qubit random circuit of the bench's recipe (U3 layers
    and brickwork CNOTs), at the default tile size."""
    gates = random_circuit(20, 10, config_seed(1))
    got = _compile_or_skip(qv, 20, 0, gates)
    assert got["passes"] == qv.qv_plan_info(20, 0, gates)["passes"]
    # the complex64 pass is built for 128 registers a thread (the next tile
    # held in registers, 4 CTAs per SM at 2^11-amplitude tiles)
    assert 0 < got["max_registers"] <= 128


def test_single_stage_relabel_pass_orders_stores_after_loads(qv):
    """A pass with one stage whose SWAP relabels change the store layout needs
    a block barrier between its loads and its stores (other warps may not have
    loaded the positions a warp stores to); one whose layout is unchanged
    stores exactly what each thread loaded and needs none."""
    swap = qv.qv_plan_source(10, 0, [Gate("swap", 6, target2=8)], 0, tile_bits=10)
    assert swap.count("__syncthreads") == 1
    u3 = qv.qv_plan_source(10, 0, [Gate("u3", 6, theta=(0.3, 0.2, 0.1))], 0, tile_bits=10)
    assert u3.count("__syncthreads") == 0
    c128 = qv.qv_plan_source(10, 1, [Gate("swap", 7, target2=9)], 0, tile_bits=10)
    assert c128.count("__syncthreads") == 1


def test_plan_source_rejects_bad_args(qv):
    g = [Gate("h", 3)]
    with pytest.raises(qv.QvError) as e:
        qv.qv_plan_source(12, 0, g, 5)
    assert e.value.status == qv.QV_ERR_ARG
    with pytest.raises(qv.QvError) as e:
        qv.qv_plan_source(12, 0, g, 0, flags=qv.QV_PLAN_INTERPRET)
    assert e.value.status == qv.QV_ERR_ARG


def test_ptxas_report_reads_every_function(tmp_path):
    """The ptxas -v report of a module with two functions: the largest register
    count counts, and a spill in either function marks the pass as spilling."""
    import subprocess
    import textwrap
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2508_15545_gb300", "csrc", "ptxas_report.h")
    src = tmp_path / "t.cpp"
    src.write_text(textwrap.dedent('''
        #include "%s"
        #include <cstdio>
        int main() {
            const std::string two =
                "ptxas info    : Compiling entry function 'helper' for 'sm_103a'\\n"
                "    0 bytes stack frame, 0 bytes spill stores, 0 bytes spill loads\\n"
                "ptxas info    : Used 40 registers, used 0 barriers\\n"
                "ptxas info    : Compiling entry function 'qv_pass' for 'sm_103a'\\n"
                "    32 bytes stack frame, 64 bytes spill stores, 32 bytes spill loads\\n"
                "ptxas info    : Used 128 registers, used 1 barriers\\n";
            const std::string clean = "    0 bytes spill stores\\nptxas info    : Used 96 registers\\n";
            std::printf("%%ld %%d %%ld %%d %%ld\\n", qv::ptxas_registers(two), int(qv::ptxas_spills(two)),
                        qv::ptxas_registers(clean), int(qv::ptxas_spills(clean)), qv::ptxas_registers("nothing"));
        }
    ''' % hdr))
    exe = tmp_path / "t"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-o", str(exe), str(src)])
    assert subprocess.check_output([str(exe)]).decode().split() == ["128", "1", "96", "0", "-1"]


def test_pure_z_tables_host(tmp_path):
    """The Pauli kernels' tables of a pure-Z group (host construction): tables
    plus the terms left out equal the term-by-term coefficient at random
    indices, for 5 to 40 qubits; every term inside one 8-bit chunk is tabled."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = tmp_path / "ztab"
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-I", os.path.join(root, "paper_2508_15545_gb300", "csrc"),
                           "-o", str(exe), os.path.join(root, "tests", "ztab_check.cu")])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    assert out[-2] == "bad 0", out
    rows = {int(l.split()[1]): l.split() for l in out if l.startswith("n ")}
    # n = 20: chunks of bits 0-7, 8-15, 16-19; the chain's 17 terms inside a chunk
    # and the identity are tabled; (7, 8) and (15, 16) are not
    assert rows[20][3] == "3" and int(rows[20][5]) >= 18
    assert rows[40][3] == "5"
