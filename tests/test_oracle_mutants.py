"""Planted mistakes in the CPU oracle must each fail a pin.

The oracle's pins (tests/test_oracle_pins.py) tie it to the paper's worked
example, closed forms, library routines and brute force.  This file checks
that those pins are strong enough: every mutant below is a copy of
oracle/hc_oracle.c with one plausible mistake planted (a dropped term, a
wrong sign, an off-by-one index or weight, a transposed index, a wrong
rounding), compiled with the oracle's own flags and loaded by the pins in a
child pytest in place of oracle/liboracle.so (HC_ORACLE_LIB).  A mutant that
passes every pin is a gap in the pins and fails this test.

Mutants are chosen so that no planted mistake reads or writes outside an
array: each changes arithmetic, a weight or a bit position, never the range
of an index.  Everything runs on the CPU.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hc_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"]

# (name, what the mistake is, [(text in hc_oracle.c, replacement), ...])
MUTANTS = [
    # quantisation and the error bound (Section IV "Quantization", Section VI-B)
    ("round_floor", "round(t) taken as floor(t)",
     [("double r = floor(t + 0.5);", "double r = floor(t);")]),
    ("quant_eps", "quantum eps instead of 2 eps",
     [("double t = load_x(x, dtype, i) / two_eps;", "double t = load_x(x, dtype, i) / (0.5 * two_eps);")]),
    ("rel_eps_max", "relative bound scaled by max instead of the value range",
     [("if (mx > mn) eps = eb * (mx - mn);", "if (mx > mn) eps = eb * mx;")]),
    # encoder and decoder (Section IV "Encoding")
    ("sign_flip_enc", "sign bit set for positive residuals",
     [("    if (p[k] < 0) {", "    if (p[k] > 0) {")]),
    ("msb_first_enc", "magnitudes written most-significant bit first",
     [("int64_t bit = k * w + j; /* position", "int64_t bit = k * w + (w - 1 - j); /* position")]),
    ("msb_first_both", "most-significant bit first in writer and reader alike",
     [("int64_t bit = k * w + j; /* position", "int64_t bit = k * w + (w - 1 - j); /* position"),
      ("int64_t bit = (int64_t)k * w + j;", "int64_t bit = (int64_t)k * w + (w - 1 - j);")]),
    ("msb_first_dec", "magnitudes read most-significant bit first",
     [("int64_t bit = (int64_t)k * w + j;", "int64_t bit = (int64_t)k * w + (w - 1 - j);")]),
    ("width_floor_log2", "width floor(log2 m) instead of the bit length",
     [("while (v != 0) {", "while (v > 1) {")]),
    ("no_sign_words", "block size without its sign words",
     [("return (int64_t)(S + 31) / 32 + ((int64_t)S * w + 31) / 32;",
       "return ((int64_t)S * w + 31) / 32 + ((int64_t)S * w + 31) / 32 * 0 + (S > 32 ? 1 : 0);")]),
    ("sign_ignored_dec", "reader drops the sign",
     [("int neg = (s[sbyte] >> (k % 8)) & 1u;", "int neg = 0 & (s[sbyte] >> (k % 8));")]),
    # in-block delta (Section IV "Decorrelation") and its stages
    ("delta_sign", "residual q_{k-1} - q_k",
     [("p[k] = q[first + k] - q[first + k - 1];", "p[k] = q[first + k - 1] - q[first + k];")]),
    ("recorrelate_drop", "recorrelation forgets the running code",
     [("q = q + p[k];", "q = head + p[k];")]),
    ("dp_head_slot", "D_p without the head in the block's first slot",
     [("dp[first] = head;", "dp[first] = 0;")]),
    # HSZx block mean (Section IV "HSZx", the worked example)
    ("mean_ties_away", "block mean with ties away from zero",
     [("i128 r = (2 * m + d - 1) / (2 * (i128)d);", "i128 r = (2 * m + d) / (2 * (i128)d);")]),
    ("mean_trunc", "block mean truncated instead of nearest",
     [("i128 r = (2 * m + d - 1) / (2 * (i128)d);", "i128 r = (2 * m) / (2 * (i128)d);")]),
    ("hszx_padded_size", "block mean over the padded size S",
     [("head = (int32_t)nearest_ratio(sum, Sb);", "head = (int32_t)nearest_ratio(sum, S);")]),
    ("hszx_resid_sign", "HSZx residual M_b - q",
     [("p[k] = q[first + k] - head;", "p[k] = head - q[first + k];")]),
    ("hszx_dq_no_mean", "HSZx D_q without the block mean",
     [("for (int64_t k = 0; k < Sb; k++) dq[first + k] = head + p[k];",
       "for (int64_t k = 0; k < Sb; k++) dq[first + k] = p[k];")]),
    # global predictors (Section IV "HSZp", "HSZp-nd"; Algorithm 4)
    ("lorenzo_term_sign", "last Lorenzo term with the wrong sign",
     [("code_at(q, L, z - 1, y - 1, x) - code_at(q, L, z - 1, y - 1, x - 1)",
       "code_at(q, L, z - 1, y - 1, x) + code_at(q, L, z - 1, y - 1, x - 1)")]),
    ("rebuild_no_plane", "rebuild without the plane below",
     [("int64_t below = z > 0 ? a[i - L[1] * L[2]] : 0;", "int64_t below = 0 * (z > 0);")]),
    ("rebuild_row", "rebuild without the row prefix",
     [("pref += a[i];", "pref = a[i];")]),
    ("lorenzo_mean_weight", "mean weight (L2 - x - 1)",
     [("t += (i128)dp[i] * (L[0] - z) * (L[1] - y) * (L[2] - x);",
       "t += (i128)dp[i] * (L[0] - z) * (L[1] - y) * (L[2] - x - 1);")]),
    ("lorenzo_var_no_plane", "Algorithm 4 without the plane below",
     [("int64_t qv = below[y * L[2] + x] + col[x];", "int64_t qv = col[x] + 0 * below[y * L[2] + x];")]),
    ("lorenzo_deriv_edge", "stage-2 derivative edge not doubled",
     [("r = 2 * dp_at(dp, L, nx[0], nx[1], nx[2]);", "r = dp_at(dp, L, nx[0], nx[1], nx[2]);")]),
    ("lorenzo_deriv_term", "stage-2 derivative drops p(i)",
     [("r = dp_at(dp, L, z, y, x) + dp_at(dp, L, nx[0], nx[1], nx[2]);",
       "r = dp_at(dp, L, nx[0], nx[1], nx[2]);")]),
    ("lorenzo_deriv_axes", "stage-2 derivative sums along its own axis too",
     [("if (ax != axis) prefix_along(D, L, ax);", "prefix_along(D, L, ax);")]),
    ("lorenzo_lap_edge", "stage-2 Laplacian subtracts at the low edge",
     [("if (c[a] > 0) v -= dp_at(dp, L, z, y, x);", "v -= dp_at(dp, L, z, y, x);")]),
    # HSZx-nd (Section IV "HSZx-nd"; Sections V-A, V-B)
    ("nd_slot_axis", "slot index along x taken modulo b0",
     [("c[2] = s % bd[2];", "c[2] = s % (bd[0] < bd[2] ? bd[0] : bd[2]);")]),
    ("nd_padded_size", "box size without clipping",
     [("n *= rest < bd[a] ? rest : bd[a];", "n *= bd[a] + 0 * rest;")]),
    ("nd_mean_padded", "box mean over the padded size",
     [("int32_t M = (int32_t)nearest_ratio(sum, Sb);", "int32_t M = (int32_t)nearest_ratio(sum, S);")]),
    ("nd_dq_no_mean", "HSZx-nd D_q without the box mean",
     [("if (i >= 0) c->out[i] = c->add_mean ? head + p[k] : p[k];",
       "if (i >= 0) c->out[i] = c->add_mean ? p[k] : p[k];")]),
    ("nd_std_uncentred", "HSZx-nd sigma not centred on mu~",
     [("int64_t d = (int64_t)dp[i] + M[nd_box_of(dims3, bd, z, y, x)] - mu;",
       "int64_t d = (int64_t)dp[i] + M[nd_box_of(dims3, bd, z, y, x)] - 0 * mu;")]),
    ("nd_mean_p_no_p", "HSZx-nd stage-2 mean without the residuals",
     [("for (int64_t i = 0; i < n; i++) t += dp[i];", "for (int64_t i = 0; i < n; i++) t += 0 * dp[i];")]),
    ("nd_deriv_border", "HSZx-nd derivative without the border correction",
     [("v += xnd_m(M, d, bd, hi) - xnd_m(M, d, bd, lo);", "v += 0 * (xnd_m(M, d, bd, hi) - xnd_m(M, d, bd, lo));")]),
    ("nd_lap_border_sign", "HSZx-nd Laplacian border correction with the wrong sign",
     [("v += xnd_m(M, d, bd, nb) - mc;", "v += mc - xnd_m(M, d, bd, nb);")]),
    # statistics (Section V-A; Eq. var, Eq. var_q, Eq. mean_m)
    ("mean_p_weight", "stage-2 mean weight (S_b - i)",
     [("total += (Sb - i + 1) * (int64_t)dp[first + i - 1];", "total += (Sb - i) * (int64_t)dp[first + i - 1];")]),
    ("eta_sum_p", "stage-2 sum of p instead of eta",
     [("a += eta;", "a += dp[first + i];")]),
    ("var_population", "variance over N instead of N - 1",
     [("double den = (double)n * (double)(n - 1);", "double den = (double)n * (double)n;")]),
    ("var_num_sign", "variance numerator N s2 + s1^2",
     [("i128 num = (i128)n * (i128)s2 - (i128)s1 * (i128)s1;", "i128 num = (i128)n * (i128)s2 + (i128)s1 * (i128)s1;")]),
    ("mean_scale", "mean scaled by eps instead of 2 eps",
     [("*mean = ((double)s1 / (double)n) * two_eps;", "*mean = ((double)s1 / (double)n) * (0.5 * two_eps);")]),
    ("sum_sq_abs", "sum of |q| instead of q^2",
     [("b += (u128)((int64_t)q[i] * (int64_t)q[i]);", "b += (u128)((int64_t)q[i] < 0 ? -(int64_t)q[i] : q[i]);")]),
    ("mean_m_padded", "Eq. mean_m with the padded size",
     [("t += (int64_t)M[b] * Sb;", "t += (int64_t)M[b] * S;")]),
    ("mean_p_x_no_mean", "HSZx stage-2 mean without M_b S_b",
     [("total += (int64_t)M[b] * Sb;", "total += 0 * (int64_t)M[b] * Sb;")]),
    ("std_x_no_mean", "HSZx sigma without M_b",
     [("int64_t d = (int64_t)dp[first + k] + M[b] - mt;", "int64_t d = (int64_t)dp[first + k] - mt;")]),
    ("mu_tilde_trunc", "mu~ truncated",
     [("int64_t mt = nearest_ratio(T, n);", "int64_t mt = T / n;")]),
    ("nd_mu_trunc", "HSZx-nd mu~ truncated",
     [("int64_t mu = nearest_ratio(T, n);", "int64_t mu = T / n;")]),
    ("std_x_population", "HSZx sigma over N",
     [("*sigma = n < 2 ? NAN : sqrt((double)ss / (double)(n - 1)) * (2.0 * eps);",
       "*sigma = n < 2 ? NAN : sqrt((double)ss / (double)n) * (2.0 * eps);")]),
    ("nd_sigma_scale", "HSZx-nd sigma scaled by eps",
     [("*sigma = sqrt(v) * 2.0 * eps;", "*sigma = sqrt(v) * eps;")]),
    ("lorenzo_var_s1", "Algorithm 4's s1 from the column buffer only",
     [("a += qv;", "a += col[x];")]),
    ("stats_f_population", "generic-flow variance over N",
     [("*var = (s + c) / (double)(n - 1);", "*var = (s + c) / (double)n;")]),
    ("dequant_f32_in_double", "float32 D_f rounded from the double product",
     [("o[i] = qf * te;", "o[i] = (float)((double)q[i] * two_eps + 0.0 * qf * te);")]),
    ("const_field_eps", "constant field gives eps = 0",
     [("if (mx > mn) eps", "if (mx >= mn) eps")]),
    ("chunk_index_end", "chunk index ends one word late",
     [("put_u64(out, h.off_chunks + 8 * h.nchunks, (uint64_t)word);",
       "put_u64(out, h.off_chunks + 8 * h.nchunks, (uint64_t)word + 1);")]),
    ("chunk_blocks_half", "chunks of 2048 codes",
     [("int64_t g = ORC_CHUNK_ELEMS / S;", "int64_t g = ORC_CHUNK_ELEMS / 2 / S;")]),
    ("heads_unaligned", "heads section not 16-byte aligned",
     [("h->off_heads = align16(h->off_widths + h->nb);", "h->off_heads = h->off_widths + h->nb;")]),
    ("dequant_scale", "f64 dequantisation by eps",
     [("o[i] = (double)q[i] * two_eps;", "o[i] = (double)q[i] * (0.5 * two_eps);")]),
    # stencils (Section V-B, V-C; Eq. derivatives, Eq. laplacian_Dq)
    ("deriv_edge_half", "one-sided edge not doubled",
     [("return 2 * ((int64_t)q[idx3(d, hi[0], hi[1], hi[2])] - q[idx3(d, i0, i1, i2)]);",
       "return ((int64_t)q[idx3(d, hi[0], hi[1], hi[2])] - q[idx3(d, i0, i1, i2)]);")]),
    ("deriv_swap", "central difference q[i-1] - q[i+1]",
     [("return (int64_t)q[idx3(d, hi[0], hi[1], hi[2])] - q[idx3(d, lo[0], lo[1], lo[2])];",
       "return (int64_t)q[idx3(d, lo[0], lo[1], lo[2])] - q[idx3(d, hi[0], hi[1], hi[2])];")]),
    ("lap_centre", "Laplacian centre weight 1 instead of 2",
     [("- 2 * center;", "- center;")]),
    ("lap_scale", "Laplacian scaled by eps instead of 2 eps",
     [("out[i] = (double)t[i] * (2.0 * eps);", "out[i] = (double)t[i] * eps;")]),
    ("lap_at_scale", "sampled Laplacian scaled by eps",
     [("val[k] = (double)num[k] * (2.0 * eps);", "val[k] = (double)num[k] * eps;")]),
    ("at_gradmag_sum", "sampled gradient magnitude from sum |D|",
     [("acc += (u128)u * u;", "acc += (u128)u * 1;")]),
    ("at_deriv_scale", "sampled derivative scaled by 2 eps",
     [("val[k] = (double)num[k] * eps;", "val[k] = (double)num[k] * 2.0 * eps;")]),
    ("gradmag_sum", "gradient magnitude from sum |D| instead of sum D^2",
     [("acc[i] += (u128)m * m;", "acc[i] += (u128)m * 1;")]),
    ("div_one_axis", "divergence differentiates every component along the first axis",
     [("int64_t D = deriv_num(q[c], d, i0, i1, i2, axes[c]);", "int64_t D = deriv_num(q[c], d, i0, i1, i2, axes[0]);")]),
    ("curl_sign", "curl dv - du",
     [("num[idx3(d, i0, i1, i2)] = du - dv;", "num[idx3(d, i0, i1, i2)] = dv - du;")]),
    ("plain_deriv_half", "generic-flow central difference not halved",
     [("g[a] = (vp - vm) / 2.0;", "g[a] = vp - vm;")]),
    ("plain_edge_half", "generic-flow one-sided edge halved",
     [("g[a] = vp - vm; /* one-sided", "g[a] = (vp - vm) / 2.0; /* one-sided")]),
    ("plain_lap_centre", "generic-flow Laplacian centre weight 1",
     [("lap += vm + vp - 2.0 * center;", "lap += vm + vp - center;")]),
    # second batch: bounds of mixed components, edges, carried state, box order
    ('div_mixed_eps', 'divergence of mixed bounds scales every term by the first eps',
     [('v += (double)D * eps[c];', 'v += (double)D * eps[0];')]),
    ('curl_mixed_eps', 'curl of mixed bounds with the bounds swapped',
     [('(double)du * eps_u - (double)dv * eps_v', '(double)du * eps_v - (double)dv * eps_u')]),
    ('plain_gradmag_2d', 'generic-flow gradient magnitude without the last axis',
     [('r = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);', 'r = sqrt(g[0] * g[0] + g[1] * g[1] + 0 * g[2]);')]),
    ('lorenzo_lap_hi_edge', 'stage-2 Laplacian drops the neighbour next to the high edge',
     [('if (c[a] < L[a] - 1) v += dp_at(dp, L, nx[0], nx[1], nx[2]);', 'if (c[a] < L[a] - 2) v += dp_at(dp, L, nx[0], nx[1], nx[2]);')]),
    ('lorenzo_deriv_hi_edge', 'stage-2 derivative high edge not doubled',
     [('r = 2 * dp_at(dp, L, z, y, x);', 'r = dp_at(dp, L, z, y, x);')]),
    ('eta_no_restart', 'eta carried across blocks',
     [('int64_t eta = 0;', 'static int64_t eta; eta = first ? eta : 0;')]),
    ('eta_s2', "eta's square taken from p",
     [('b += (u128)(eta * eta);', 'b += (u128)(eta * dp[first + i]);')]),
    ('hszp_as_nd', "HSZp predicts over the field's axes",
     [('if (pred == 3) {', 'if (pred == 99) {')]),
    ('nd_box_order', 'boxes stored with axes 1 and 2 transposed',
     [('G->k[2] = b % G->g[2];', 'G->k[2] = (b / G->g[1]) % G->g[2];'),
      ('G->k[1] = (b / G->g[2]) % G->g[1];', 'G->k[1] = b % G->g[1];')]),
    ('nd_mean_m_unweighted', 'HSZx-nd Eq. mean_m without the box sizes',
     [('t += (int64_t)M[b] * nd_box_size(dims3, bd, b);', 't += (int64_t)M[b] * 1 + 0 * nd_box_size(dims3, bd, b);')]),
    ('nd_deriv_lo_edge', 'HSZx-nd derivative low edge not doubled',
     [('          hi[axis] = 1;\n          e = 2;', '          hi[axis] = 1;\n          e = 1;')]),
    ('header_eps_eb', 'header stores eb in place of eps',
     [('put_f64(out, 40, eps);', 'put_f64(out, 40, eb);')]),
    ('rel_min_first', 'value range from the first element',
     [('if (v < mn) mn = v;', 'if (v < mn) mn = mn;')]),
    ('sd_is_var', 'standard deviation without the root',
     [('*sd = sqrt(*var);', '*sd = *var;')]),
    ('lorenzo_var_s2', "Algorithm 4's s2 from the column buffer",
     [('b += (u128)(qv * qv);', 'b += (u128)(qv * col[x]);')]),
    # third batch: header fields, limits and the reader's structural checks (none that
    # guards memory is dropped)
    ('header_wmax', 'header max width one too high',
     [('put_u32(out, 136, (uint32_t)wmax);', 'put_u32(out, 136, (uint32_t)wmax + 1u);')]),
    ('header_qmax', 'header max |q| one too high',
     [('put_u32(out, 60, (uint32_t)qmax);', 'put_u32(out, 60, (uint32_t)qmax + 1u);')]),
    ('header_eb_mode', 'header bound mode always absolute',
     [('put_u32(out, 56, (uint32_t)eb_mode);', 'put_u32(out, 56, 0u * (uint32_t)eb_mode);')]),
    ('header_eb_is_eps', 'header stores eps in place of eb',
     [('put_f64(out, 48, eb);', 'put_f64(out, 48, eps);')]),
    ('header_ndim_3', 'header ndim always 3',
     [('put_u8(out, 7, (uint32_t)ndim);', 'put_u8(out, 7, 3u + 0u * (uint32_t)ndim);')]),
    ('stats_f_mean_n1', 'generic-flow mean over N + 1',
     [('double mu = (s + c) / (double)n;', 'double mu = (s + c) / (double)(n + 1);')]),
    ('qlimit_2x', 'codes accepted up to 2^31',
     [('if (!(fabs(r) < (double)ORC_QLIMIT)) return ORC_ERR_RANGE;', 'if (!(fabs(r) < 2.0 * (double)ORC_QLIMIT)) return ORC_ERR_RANGE;')]),
    ('resid_range_30', 'global residuals limited to 2^30',
     [('if (v <= -((int64_t)1 << 31) || v >= ((int64_t)1 << 31)) {', 'if (v <= -((int64_t)1 << 30) || v >= ((int64_t)1 << 30)) {')]),
    ('chunk_check_dropped', 'reader ignores the chunk index',
     [('if (b % h.G == 0 && (int64_t)get_u64(s, h.off_chunks + 8 * (b / h.G)) != word) {', 'if (b % h.G == 0 && (int64_t)get_u64(s, h.off_chunks + 8 * (b / h.G)) != word && 0) {')]),
    ('magic_check_dropped', 'reader ignores magic and version',
     [('if (get_u32(s, 0) != ORC_MAGIC || get_u16(s, 4) != ORC_VERSION) return ORC_ERR_CORRUPT;', 'if (0 && (get_u32(s, 0) != ORC_MAGIC || get_u16(s, 4) != ORC_VERSION)) return ORC_ERR_CORRUPT;')]),
    ('payload_total_check', 'reader ignores the payload total of the walk',
     [('if (word != h.payload_words ||', 'if (0 * (word != h.payload_words) ||')]),
    ('global_heads_allowed', 'stage 1 of a global-predictor stream not refused',
     [('if (h.pred == 2 || h.pred == 3) return ORC_ERR_UNSUPPORTED;', 'if (0 * h.pred) return ORC_ERR_UNSUPPORTED;')]),
    ('msb_in_byte_both', 'bits taken most-significant first inside each byte, writer and reader alike',
     [('out[byte] |= (uint8_t)(1u << (bit % 8));', 'out[byte] |= (uint8_t)(1u << (7 - bit % 8));'),
      ('if ((s[byte] >> (bit % 8)) & 1u) m |= 1u << j;', 'if ((s[byte] >> (7 - bit % 8)) & 1u) m |= 1u << j;')]),
]


def _mutate(src, edits):
    for old, new in edits:
        assert src.count(old) == 1, f"mutation site must occur once in hc_oracle.c: {old!r}"
        src = src.replace(old, new)
    return src


def _run_pins(lib_path):
    env = dict(os.environ, HC_ORACLE_LIB=lib_path, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def _build_and_pin(tmpdir, name, edits):
    src = _mutate(open(SRC).read(), edits)
    c_path = os.path.join(tmpdir, f"{name}.c")
    so_path = os.path.join(tmpdir, f"lib{name}.so")
    with open(c_path, "w") as f:
        f.write(src)
    cc = subprocess.run(["gcc", *CFLAGS, "-o", so_path, c_path, "-lm"], capture_output=True, text=True)
    assert cc.returncode == 0, f"{name}: the mutant does not compile:\n{cc.stderr}"
    return _run_pins(so_path)


def test_mutant_sites_unique():
    src = open(SRC).read()
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))
    for name, _, edits in MUTANTS:
        _mutate(src, edits)


def test_every_planted_mistake_fails_a_pin(tmp_path):
    tmpdir = str(tmp_path)
    # the unmodified source through the same harness passes every pin
    rc, out = _build_and_pin(tmpdir, "control", [])
    assert rc == 0, f"the unmodified oracle fails its pins through the harness:\n{out}"
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {m[0]: ex.submit(_build_and_pin, tmpdir, m[0], m[2]) for m in MUTANTS}
        results = {k: f.result() for k, f in futs.items()}
    survivors = [(name, what) for name, what, _ in MUTANTS if results[name][0] == 0]
    # a pin failure is exit status 1; anything else (a collection error or a
    # crash) would mean the harness, not a pin, stopped the mutant
    odd = {name: rc for name, (rc, _) in results.items() if rc not in (0, 1)}
    assert not odd, f"mutants stopped by something other than a failing pin: {odd}"
    assert not survivors, f"planted mistakes that no pin catches: {survivors}"
