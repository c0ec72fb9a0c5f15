"""Planted mistakes: the oracle's pins must catch every one of them.

Each mutant is a copy of the oracle's C source with one plausible mistake:
a dropped term, a wrong index, sign or shift, a transposed operand.  The pin
tests (test_oracle_hash.py, test_oracle_update.py, test_oracle_close.py) run
in a child process against that copy (SD_ORACLE_SRC) and at least one must
fail.  An unmodified copy runs first as the control: every pin passes.

Not planted: changes that are themselves a valid reading of the paper (another
odd multiplier, the additive constant of H1, another seed derivation), which
the pins leave open by design and the GPU parity tests fix, and changes that
cannot alter any result (z_0 <= Zmin for z_0 < Zmin: Zmin is not an integer).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_SRC = os.path.join(ROOT, "oracle", "sd_oracle.c")
PIN_FILES = ["tests/test_oracle_hash.py", "tests/test_oracle_update.py", "tests/test_oracle_close.py"]

# name -> (what it breaks, [(text, replacement), ...]); each text occurs once
MUTANTS = {
    "splitmix64-shift": ("the published generator", [
        ("z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;")]),
    "same-constants-both-directions": ("one hash group per direction", [
        ("0x9E3779B97F4A7C15ull * (uint64_t)(dir + 1u)", "0x9E3779B97F4A7C15ull")]),
    "dh0-low-bits": ("DH_0 as multiply-shift (top k bits)", [
        ("return (uint32_t)(A0 * x) >> (32u - k);", "return (uint32_t)(A0 * x) & ((1u << k) - 1u);")]),
    "eq2-block-index": ("Eq. 2: block i starts at bit (i-1) alpha", [
        ("s = (i - 1u) * alpha;", "s = i * alpha;")]),
    "eq2-drops-dh0": ("Eq. 2: the block is xored with DH_0", [
        ("return blk ^ h0;", "return blk;")]),
    "eq2-mask-short": ("Eq. 2: blocks of k bits", [
        ("blk = (s >= 32u) ? 0u : ((x >> s) & ((1u << k) - 1u));",
         "blk = (s >= 32u) ? 0u : ((x >> s) & ((1u << (k - 1u)) - 1u));")]),
    "eq2-shift-wraps": ("Eq. 2: bits past 31 are zero", [
        ("blk = (s >= 32u) ? 0u : ((x >> s) & ((1u << k) - 1u));",
         "blk = (x >> (s & 31u)) & ((1u << k) - 1u);")]),
    "h1-low-bits": ("H1 as multiply-add-shift (top log2 g bits)", [
        ("return (uint32_t)((A1 * (uint64_t)y + B1) >> (64u - log2u(g)));",
         "return (uint32_t)((A1 * (uint64_t)y + B1) & (uint64_t)(g - 1u));")]),
    "update-key-transposed": ("Algorithm 1: direction 0 keys on the source", [
        ("uint32_t a0 = dir == 0 ? src : dst;", "uint32_t a0 = dir == 0 ? dst : src;")]),
    "update-skips-last-row": ("Algorithm 1: one bit in every row", [
        ("for (uint32_t i = 0; i < p->r; i++) {\n                uint32_t LEidx",
         "for (uint32_t i = 0; i + 1u < p->r; i++) {\n                uint32_t LEidx")]),
    "update-bit-in-wrong-word": ("Algorithm 1: bit BITidx of the estimator", [
        ("LEp[BITidx >> 5] |= 1u << (BITidx & 31u);", "LEp[0] |= 1u << (BITidx & 31u);")]),
    "z0-counts-ones": ("z_0 = zero bits of an estimator", [
        ("uint32_t z = p->g - weight(", "uint32_t z = weight(")]),
    "zmin-exponent-sign": ("Zmin = g e^(-theta/g)", [
        ("return (double)g * exp(-theta / (double)g);", "return (double)g * exp(theta / (double)g) / 8.0;")]),
    "zmin-drops-g": ("Zmin = g e^(-theta/g)", [
        ("return (double)g * exp(-theta / (double)g);", "return exp(-theta / (double)g);")]),
    "psi-no-row-average": ("w' is the mean of the rows' w(i)'", [
        ("w = wsum / (double)p->r;", "w = wsum;")]),
    "psi-drops-one-minus": ("Lemma 1: psi = 1 - e^(-w/(g 2^k))", [
        ("return 1.0 - exp(-w / G);", "return exp(-w / G);")]),
    "psi-per-estimator-size": ("Lemma 1 over all g 2^k bits of a row", [
        ("double G = (double)p->g * (double)((uint64_t)1 << p->k);", "double G = (double)p->g;")]),
    "eq4-exponent-r-minus-1": ("Eq. 4: psi^r", [
        ("pow(psi, (double)r)", "pow(psi, (double)(r - 1u))")]),
    "eq4-denominator-sign": ("Eq. 4: g - g psi^r", [
        ("(gd - gd * pow(psi, (double)r))", "(gd + gd * pow(psi, (double)r))")]),
    "eq4-sign": ("Eq. 4: C = -g ln(...)", [
        ("return -gd * log(", "return gd * log(")]),
    "ule-or-not-and": ("Definition 1: ULE is the AND of the r estimators", [
        ("uint32_t ule = 0xFFFFFFFFu;", "uint32_t ule = 0u;"), ("ule &= cell_ptr", "ule |= cell_ptr")]),
    "sz-counts-ones": ("SZ = zero bits of ULE", [("return p->g - ones;", "return ones;")]),
    "join-overlap-transposed": ("Algorithm 3: high k-alpha bits of BL(1) = low k-alpha of BL(2)", [
        ("if ((blk1 >> al) != (blk2 & ovmask)) continue;", "if ((blk1 & ovmask) != (blk2 >> al)) continue;")]),
    "join-new-bits-at-alpha": ("Algorithm 3: BL(2)'s new bits go to bit k", [
        ("else { if (k + al > 32u && (add >> (32u - k))) continue; hi = add << k; }",
         "else { if (k + al > 32u && (add >> (32u - k))) continue; hi = add << al; }")]),
    "join-stage-offset": ("Algorithm 4: stage i adds bits from (i-2) alpha + k", [
        ("uint32_t pos = (i - 2u) * al + k;", "uint32_t pos = (i - 1u) * al + k;")]),
    "join-without-dh0-check": ("the restored a0 must hash to its CL_0", [
        ("if (dh0(h.A0[dir], k, sub[s]) == scl[s]) emit(out, cap, &count, sub[s]);",
         "emit(out, cap, &count, sub[s]);")]),
    "preimage-operands-transposed": ("DH_0 preimages: CL_0 is the top k bits", [
        ("uint32_t a = A0inv * (((uint32_t)c << (32u - k)) | (uint32_t)t);",
         "uint32_t a = A0inv * (((uint32_t)t << k) | (uint32_t)c);")]),
    "inverse-short-newton": ("A0^-1 mod 2^32 (five Newton steps from 3 bits)", [
        ("for (int s = 0; s < 5; s++) x *= 2u - A * x;", "for (int s = 0; s < 3; s++) x *= 2u - A * x;")]),
    "report-keeps-below-theta": ("report C(a0) >= theta", [
        ("if (C < p->theta) continue;", "if (C >= p->theta) continue;")]),
    "saturation-ignored": ("a row with ZR(i) = 0 has no psi", [
        ("if (zr[i] == 0) return -1.0;", "if (zr[i] == 0) continue;")]),
    "overload-cap-off-by-one": ("pair_cap bounds |HE(0)| 2^(32-k)", [
        ("<< (32u - p->k)) > p->pair_cap)", "<< (32u - p->k)) > p->pair_cap + 1u)")]),
    "overload-bound-uses-k-bits": ("the work bound counts the 2^(32-k) preimages of each hot c0", [
        ("<< (32u - p->k)) > p->pair_cap)", "<< p->k) > p->pair_cap)")]),
    "overloaded-k-counted-exactly": ("an overloaded |K| is reported as cand_cap + 1", [
        ("            if (count > cap) goto done;\n", "")]),
    "cand-cap-off-by-one": ("cand_cap bounds |K|", [
        ("if (nk > kcap) { sum->flags[dir] |= OR_FLAG_OVERLOAD_CANDS; continue; }",
         "if (nk >= kcap) { sum->flags[dir] |= OR_FLAG_OVERLOAD_CANDS; continue; }")]),
    "update-break-not-continue": ("Algorithm 1: a bit already set skips only its own row", [
        ("if ((LEp[BITidx >> 5] >> (BITidx & 31u)) & 1u) continue;",
         "if ((LEp[BITidx >> 5] >> (BITidx & 31u)) & 1u) break;")]),
    "h1-hashes-the-key": ("Algorithm 1: the bit comes from the peer", [
        ("uint32_t BITidx = or_h1(h.A1[dir], h.B1[dir], p->g, b0);",
         "uint32_t BITidx = or_h1(h.A1[dir], h.B1[dir], p->g, a0);")]),
    "inbound-hashes-dst": ("direction 1 counts a destination's sources", [
        ("uint32_t b0 = dir == 0 ? dst : src;", "uint32_t b0 = dst;")]),
    "row-stats-reads-row-0": ("z_0 of every row's own estimators", [
        ("uint32_t z = p->g - weight(cell_ptr(p, (uint32_t *)grid, dir, i, j), p->g);",
         "uint32_t z = p->g - weight(cell_ptr(p, (uint32_t *)grid, dir, 0, j), p->g);")]),
    "zr-keeps-last-estimator": ("ZR(i) sums z_0 over the row", [("            zr[i] += z;", "            zr[i] = z;")]),
    "hot-sets-read-row-0": ("HE(i) from row i's z_0", [
        ("if ((double)z0[(uint64_t)i * ncell + j] < Zmin) he[(uint64_t)i * ncell + nhe[i]++] = j;",
         "if ((double)z0[j] < Zmin) he[(uint64_t)i * ncell + nhe[i]++] = j;")]),
    "zmin-theta-over-2g": ("Zmin = g e^(-theta/g)", [
        ("return (double)g * exp(-theta / (double)g);", "return (double)g * exp(-theta / (2.0 * (double)g));")]),
    "psi-log-inverted": ("w(i)' = -g 2^k ln(ZR(i) / (g 2^k))", [
        ("wi = -G * log((double)zr[i] / G);", "wi = -G * log(G / (double)zr[i]);")]),
    "psi-first-row-only": ("w' averages all r rows", [
        ("        wsum += wi;", "        wsum += (i == 0) ? wi * p->r : 0.0;")]),
    "eq4-sz-off-by-one": ("Eq. 4 takes SZ itself", [
        ("return -gd * log((double)sz / (", "return -gd * log((double)(sz + 1u) / (")]),
    "sz-half-the-words": ("SZ over all g bits of ULE", [
        ("    for (uint32_t q = 0; q < p->g / 32u; q++) {\n        uint32_t ule",
         "    for (uint32_t q = 0; q < p->g / 64u; q++) {\n        uint32_t ule")]),
    "join-mask-one-bit-wide": ("Algorithm 3: overlaps of k - alpha bits", [
        ("uint32_t ovmask = (ov == 32u) ? 0xFFFFFFFFu : ((1u << ov) - 1u);",
         "uint32_t ovmask = (ov == 32u) ? 0xFFFFFFFFu : ((2u << ov) - 1u);")]),
    "join-stage-overlap-index": ("Algorithm 4: BL(i) overlaps the partial from bit (i-1) alpha", [
        ("uint32_t top = (i - 1u) * al;", "uint32_t top = (i - 2u) * al;")]),
    "join-wraps-past-bit-31": ("Algorithm 3: a0 has 32 bits", [
        ("else { if (k + al > 32u && (add >> (32u - k))) continue; hi = add << k; }",
         "else { hi = add << k; }")]),
    "join-stage-wraps-past-bit-31": ("Algorithm 4: a0 has 32 bits", [
        ("else { if (pos + al > 32u && (add >> (32u - pos))) continue; hi = add << pos; }",
         "else { hi = add << pos; }")]),
    "preimage-skips-row-1": ("K needs every row hot", [
        ("for (uint32_t i = 1; i < p->r && all; i++)\n                all = hot[(uint64_t)i * ncell + dh(h.A0[dir], k, p->alpha, i, a)];",
         "for (uint32_t i = 2; i < p->r && all; i++)\n                all = hot[(uint64_t)i * ncell + dh(h.A0[dir], k, p->alpha, i, a)];")]),
}


def _mutant_source(name):
    with open(ORACLE_SRC) as f:
        src = f.read()
    for old, new in MUTANTS[name][1]:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    return src


def _run_pins(src_path, timeout=900):
    env = dict(os.environ, SD_ORACLE_SRC=src_path)
    cmd = [sys.executable, "-m", "pytest", *PIN_FILES, "-x", "-q", "-p", "no:cacheprovider",
           "-m", "not gpu"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_every_mutant_applies_and_compiles(tmp_path):
    for name in MUTANTS:
        path = tmp_path / f"{name}.c"
        path.write_text(_mutant_source(name))
        subprocess.run(["gcc", "-fsyntax-only", "-std=c11", str(path)], check=True)


@pytest.mark.slow
def test_pins_catch_every_planted_mistake(tmp_path):
    jobs = {"control": open(ORACLE_SRC).read()}
    jobs.update({name: _mutant_source(name) for name in MUTANTS})
    paths = {}
    for name, src in jobs.items():
        d = tmp_path / name
        d.mkdir()
        (d / "sd_oracle.c").write_text(src)
        paths[name] = str(d / "sd_oracle.c")
    with ThreadPoolExecutor(max_workers=max(2, min(16, os.cpu_count() or 2))) as ex:
        res = dict(zip(paths, ex.map(_run_pins, paths.values())))

    control = res.pop("control")
    assert control.returncode == 0, control.stdout[-3000:] + control.stderr[-3000:]
    survived = [n for n, r in res.items() if r.returncode == 0]
    assert not survived, f"mutants no pin catches: {survived}"
    # caught by a failing pin (or a crash of the mutant), not by a harness error
    for name, r in res.items():
        tail = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
        assert r.returncode < 0 or (r.returncode == 1 and " failed" in tail), (name, r.returncode,
                                                                                r.stdout[-2000:],
                                                                                r.stderr[-2000:])
