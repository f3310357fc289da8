"""The committed per-order kernel lists (csrc/apply3d_p{2..9}.cu) are the output
of their generator, csrc/gen_orders.py, so that a candidate table edited in one
place cannot silently disagree with the compiled lists (CPU only)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1809_05471_gb300", "csrc")


def test_order_lists_are_the_generator_output(tmp_path):
    spec = importlib.util.spec_from_file_location("gen_orders", os.path.join(CSRC, "gen_orders.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    gen.generate(str(tmp_path))
    for p in range(2, 10):
        name = "apply3d_p%d.cu" % p
        want = (tmp_path / name).read_text()
        with open(os.path.join(CSRC, name)) as f:
            assert f.read() == want, name + " differs from gen_orders.py's output"


def test_persistent_batch_tiles_are_compiled_candidates():
    # the persistent batch schedule runs the register-prefetch kernel of each order
    # at a fixed tile; plans of that tile must be buildable in every precision the
    # schedule takes (host-only queries: no device is touched)
    from paper_1809_05471_gb300 import build
    from paper_1809_05471_gb300 import igasf as G
    build.build()
    for prec in (G.FP32, G.BF16):
        for p in range(2, 7):
            tile = list(G.batch_persistent_tile(p, prec))
            cands = [(list(t), v) for t, v in G.list_kernels(3, p, prec)]
            assert (tile, G.KERNEL_REGISTERS) in cands, (prec, p, tile, cands)
