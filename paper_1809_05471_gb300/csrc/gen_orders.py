"""Writes csrc/apply3d_p{2..9}.cu, the per-order lists of compiled 3D tile
kernels: the FP64 kernel, the FP32/BF16 candidates (first = default, chosen by
timing sweeps on the order-sweep workload, about 2M dofs), the shapes the
IGASF_TILE_SEARCH build adds, and the two on-the-fly candidates.

A candidate is (variant, tile[, register cap in resident blocks[, reload[, BF16
too]]]), variant R = register prefetch, T = TMA ring; the cap and the reload apply
to FP32 only unless the last flag is set; the L2 prefetch per order and precision
is in l2_prefetch; ("pair", FP32 candidate, BF16 candidate)
gives the two precisions different defaults.

The lists of p = 2 and 4 end with the paper's narrow macro-element shape, p x p x 1
elements with the thin direction last (Sec. 4, narrow macro-elements), for the
autotuner; for odd p that shape has an odd number of direction-1 points per tile,
which the pencil-pair kernels cannot hold.

    python paper_1809_05471_gb300/csrc/gen_orders.py

tests/test_generated_sources.py checks that the committed files are its output.
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))
R, T = "r", "t"
f64 = {2: "8, 8, 8", 3: "8, 4, 4", 4: "4, 4, 4", 5: "4, 2, 2", 6: "4, 2, 2", 7: "2, 2, 2", 8: "2, 2, 2", 9: "2, 1, 2"}
main = {
 2: [(R, "8, 8, 4"), (R, "8, 8, 2"), (T, "16, 8, 4"), (R, "2, 2, 1")],
 3: [("pair", (R, "8, 4, 4", 4, 1), (R, "4, 4, 8")), ("pair", (T, "8, 8, 4"), (T, "8, 8, 4")),
     ("pair", (R, "4, 4, 8"), (R, "8, 4, 4")), (R, "4, 4, 4")],
 4: [("pair", (R, "4, 4, 4", 4, 1), (R, "4, 4, 8")), ("pair", (R, "4, 4, 8", 4, 1), (R, "4, 4, 4")),
     (T, "8, 4, 2"), (T, "4, 4, 4"), (R, "4, 4, 1")],
 5: [("pair", (T, "4, 4, 4"), (R, "4, 2, 8")), (R, "4, 4, 4"), (R, "4, 2, 4"), ("pair", (R, "4, 2, 8"), (T, "4, 4, 4"))],
 6: [(R, "2, 2, 8", 4, 1, 1), (R, "2, 2, 2", 4), (R, "4, 4, 2"), (T, "4, 2, 2")],
 7: [("pair", (R, "2, 2, 8", 3, 1), (R, "2, 2, 8")), ("pair", (R, "2, 2, 6", 3, 1), (R, "2, 2, 6")),
     (T, "2, 2, 4", 0, 1), (R, "4, 2, 2")],
 8: [(R, "2, 2, 8"), (R, "2, 2, 6"), (R, "2, 2, 2"), (T, "4, 2, 1")],
 9: [("pair", (R, "2, 2, 8", 2, 1), (R, "2, 2, 6", 2, 1, 1)), ("pair", (R, "2, 2, 6", 2, 1, 1), (R, "2, 2, 8")),
     (R, "2, 2, 2", 2, 1), (T, "2, 2, 2")],
}
search = {
 2: ["8, 8, 2", "8, 8, 4", "16, 8, 4", "8, 4, 8", "8, 8, 8", "16, 8, 2"],
 3: ["8, 4, 4", "4, 4, 4", "8, 8, 4", "8, 8, 2", "4, 4, 2", "8, 4, 2"],
 4: ["4, 4, 4", "4, 2, 4", "8, 4, 4", "8, 4, 2", "2, 2, 4", "4, 4, 2"],
 5: ["4, 4, 4", "4, 2, 4", "2, 2, 4", "4, 4, 2", "2, 2, 2", "4, 2, 2"],
 6: ["2, 2, 8", "2, 2, 6", "4, 2, 4", "4, 4, 2", "2, 2, 4", "4, 2, 2", "2, 2, 2"],
 7: ["2, 2, 8", "2, 2, 6", "2, 2, 4", "4, 2, 4", "4, 2, 2", "2, 2, 2"],
 8: ["2, 2, 8", "2, 2, 6", "2, 2, 4", "2, 2, 2", "4, 2, 1"],
 9: ["2, 2, 8", "2, 2, 6", "2, 2, 4", "2, 2, 2", "2, 1, 2"],
}
geo = {  # factors on the fly: (tile, Z of all slabs up front)
 2: [("8, 8, 2", 1), ("8, 4, 4", 1)],
 3: [("8, 4, 2", 1), ("4, 4, 4", 1)],
 4: [("4, 4, 2", 1), ("4, 4, 4", 1)],
 5: [("4, 2, 2", 1), ("2, 2, 2", 1)],
 6: [("2, 2, 8", 0), ("2, 2, 2", 1)],
 7: [("2, 2, 2", 0), ("2, 2, 1", 0)],
 8: [("2, 2, 4", 0), ("2, 2, 2", 0)],
 9: [("2, 2, 4", 0), ("2, 2, 2", 0)],
}
# tensor-core kernels of IGASF_TF32 / IGASF_BF16_MMA: (tile, warps per block,
# minimum resident blocks asked of the register allocator), default first
tc = {
 2: [("8, 8, 4", 8, 2), ("8, 8, 2", 8, 2)],
 3: [("8, 4, 4", 6, 2), ("4, 4, 4", 9, 2)],
 4: [("4, 4, 4", 8, 2), ("4, 4, 8", 8, 2)],
 5: [("4, 4, 4", 5, 2), ("2, 2, 8", 7, 2)],
 6: [("2, 2, 8", 9, 2), ("4, 2, 4", 6, 2)],
 7: [("2, 2, 8", 7, 2), ("2, 2, 6", 7, 2)],
 8: [("2, 2, 8", 8, 2), ("2, 2, 6", 8, 2)],
 9: [("2, 2, 8", 7, 2), ("2, 2, 6", 7, 2)],
}
# orders whose register-prefetch kernels request their tile's factors into L2
# at entry (kL2Prefetch), per precision: where the order sweep measured a gain
# (FP32 p = 3: 0.244 -> 0.215 ms; BF16 p = 4: 0.436 -> 0.385 ms; 2 to 7 % at
# p = 7..9); off at the bench cube's p = 4 FP32, where it slowed the gather
l2_prefetch = {"fp32": {3, 7, 8, 9}, "bf16": {4, 7, 8, 9}}
# FP32 register-prefetch candidates whose mass kernel asks for more resident
# blocks than the stiffness (order, tile): blocks; the 64^3, p = 4 cube's FP32
# mass 31.0 -> 29.0 us with 6 (104 -> 80 registers, no spills; 7 and 8 blocks
# measured the same as 6)
mass_minb = {(4, "4, 4, 4"): 6, (4, "4, 4, 8"): 6}
# Tiles re-measured after phase C kept only p live values per array (2M dofs,
# stiffness, ms per apply): deeper tiles for BF16, p = 2 8x8x4 (0.084 -> 0.074;
# FP32 0.091 -> 0.085 too), p = 3 4x4x8 (0.244 -> 0.211), p = 4 4x4x8 (0.405 ->
# 0.372), p = 5 4x2x8 (1.134 -> 0.949); FP32 keeps its tiles at p = 3..5 (4x4x8 at
# p = 4 spills at 4 blocks: 0.493 -> 0.575). Caps re-measured too: p = 7 FP32
# 3 blocks instead of 2 (168 registers, 4 bytes spilled; 2M dofs 3.61 -> 3.36 ms);
# BF16 p = 6 at 5 blocks and p = 7 at 3 blocks (with reload) were slower (1.78 ->
# 1.94, 2.72 -> 2.91 ms), p = 8 spills at any cap, p = 9 at 3 blocks spills 5 KB.
# FP32 p = 7 and 9 then default to 2x2x8 (p = 7: stiffness 3.45 ms either way, mass
# 1.27 -> 1.17 ms; p = 9: stiffness 7.95 -> 7.83 ms, mass 3.03 -> 2.95 ms); BF16
# keeps 2x2x6 at p = 9 (2x2x8: 10.8 ms)
mk = {R: "make_apply3d_f32r", T: "make_apply3d_f32"}
name = {R: "register prefetch", T: "TMA ring"}
def generate(outdir=HERE):
    """Write apply3d_p{2..9}.cu into outdir."""
    for P in range(2, 10):
        L = ["// 3D apply kernels of order p = %d. FP64: scalar kernel, tile %s elements." % (P, f64[P]),
             "// FP32 (packed FP32x2) candidates, the first the default (fastest in a sweep",
             "// of tile shapes and factor-stream variants on the order-sweep workload);",
             "// BF16 (bfloat16-stored factors) uses the same candidates unless a line names both:"]
        def describe(c, bf=False):
            v, t = c[0], c[1]
            mbm = mass_minb.get((P, t), 0) if v == R and not bf else 0
            return "%s, tile %s%s%s%s%s" % (name[v], t, (", registers capped for %d resident blocks" % c[2]) if len(c) > 2 and c[2] else "",
                                           (" (mass %d, FP32)" % mbm) if mbm else "",
                                           ", tables reloaded for the transposed sweep" if len(c) > 3 and c[3] else "",
                                           " (BF16 too)" if len(c) > 4 and c[4] else "")
        for c in main[P]:
            if c[0] == "pair":
                L.append("//   FP32: %s; BF16: %s" % (describe(c[1]), describe(c[2], bf=True)))
            else:
                L.append("//   %s" % describe(c))
        L.append("// Register-prefetch kernels request their tile's factors into L2 at entry: "
                 "FP32 %s, BF16 %s." % ("yes" if P in l2_prefetch["fp32"] else "no",
                                       "yes" if P in l2_prefetch["bf16"] else "no"))
        L.append("// IGASF_TILE_SEARCH compiles every listed shape in both variants.")
        L.append("// Tensor-core kernels (IGASF_TF32, IGASF_BF16_MMA): %s." % "; ".join(
            "tile %s, %d warps" % (t, w) for t, w, _ in tc[P]))
        L.append("// Factors evaluated on the fly (FP32): tile %s first, then %s." % (geo[P][0][0], geo[P][1][0]))
        L.append('#include "apply3d.cuh"\n#include "apply3d_f32.cuh"\n#include "apply3d_f32g.cuh"\n#include "apply3d_f32r.cuh"\n#include "apply3d_tc.cuh"\n\nnamespace igasf {\n')
        L.append("int apply3d_p%d(int prec, ApplyKernel *out, int max_out) {" % P)
        L.append("  int n = 0;\n  if (prec == IGASF_FP64) {")
        L.append("    if (n < max_out) out[n++] = make_apply3d<double, %d, %s>();\n    return n;\n  }" % (P, f64[P]))
        L.append("  if (tensor_core_prec(prec)) {\n    const bool b = prec == IGASF_BF16_MMA;")
        for t, w, mb in tc[P]:
            L.append("    if (n < max_out) out[n++] = b ? make_apply3d_tc<%d, %s, TC_BF16, %d, %d>() : make_apply3d_tc<%d, %s, TC_TF32, %d, %d>();"
                     % (P, t, w, mb, P, t, w, mb))
        L.append("    return n;\n  }")
        L.append("  const bool bf = prec == IGASF_BF16;")
        L.append("#ifndef IGASF_TILE_SEARCH")
        def inst(c):
            """(BF16, FP32) instantiations of a candidate (variant, tile[, minb[, reload[, BF16 too]]])."""
            v, t = c[0], c[1]
            minb = c[2] if len(c) > 2 else 0
            reload = bool(len(c) > 3 and c[3])
            if v == R:
                f32 = (1 if reload else 0) | (2 if P in l2_prefetch["fp32"] else 0)
                if len(c) > 4 and c[4]:
                    mb16, f16 = minb, (1 if reload else 0)
                else:
                    # BF16 keeps the compiler's register choice and the tables in registers
                    # (measured faster for the bfloat16 stream at these orders)
                    mb16, f16 = 0, 0
                f16 |= 2 if P in l2_prefetch["bf16"] else 0
                mbm = mass_minb.get((P, t), 0)
                return ("%s<%d, %s, true, 2, %d, %d>()" % (mk[v], P, t, mb16, f16),
                        "%s<%d, %s, false, 2, %d, %d%s>()" % (mk[v], P, t, minb, f32,
                                                               ", %d" % mbm if mbm else ""))
            if reload:
                return ("%s<%d, %s, true, true>()" % (mk[v], P, t), "%s<%d, %s, false, true>()" % (mk[v], P, t))
            return ("%s<%d, %s, true>()" % (mk[v], P, t), "%s<%d, %s>()" % (mk[v], P, t))
        def inst2(c):
            """("pair", FP32 candidate, BF16 candidate): different defaults per precision."""
            if c[0] == "pair":
                return inst(c[2])[0], inst(c[1])[1]
            return inst(c)
        for c in main[P]:
            b16, f32 = inst2(c)
            L.append("  if (n < max_out) out[n++] = bf ? %s : %s;" % (b16, f32))
        L.append("#else")
        first = main[P][0]
        b16, f32 = inst2(first)
        L.append("  if (n < max_out) out[n++] = bf ? %s : %s;" % (b16, f32))
        firsts = [first[1][:2], first[2][:2]] if first[0] == "pair" else [tuple(first[:2])]
        for v in (R, T):
            for t in search[P]:
                if (v, t) in [tuple(f) for f in firsts]:
                    continue
                L.append("  if (n < max_out) out[n++] = bf ? %s<%d, %s, true>() : %s<%d, %s>();" % (mk[v], P, t, mk[v], P, t))
        L.append("#endif\n  return n;\n}\n")
        L.append("int apply3d_p%d_geo(ApplyKernel *out, int max_out) {\n  int n = 0;" % P)
        for t, z in geo[P]:
            L.append("  if (n < max_out) out[n++] = make_apply3d_f32g<%d, %s, %s>();" % (P, t, "true" if z else "false"))
        L.append("  return n;\n}\n\n}  // namespace igasf")
        open(os.path.join(outdir, "apply3d_p%d.cu" % P), "w").write("\n".join(L) + "\n")


if __name__ == "__main__":
    generate()
