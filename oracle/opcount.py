"""Operation count of the method from an instrumented oracle run (TEST AND MEASUREMENT
INFRASTRUCTURE: it builds and runs the oracle; the product path never uses it).

The oracle is compiled twice with its condition estimate compiled out (ORC_CONDITION=0, so
only the method's own arithmetic remains): first with GCC's profile instrumentation, which is
then run on a sample of a workload, then again with the recorded profile, dumping GCC's
optimised intermediate form (GIMPLE) with the execution count of every basic block.  Every
statement of a block is classified by its operation and the type of its result:

  fp   floating-point arithmetic, comparisons, conversions to floating point, fabs/floor/
       fmin/fmax-like operations;
  int  integer and boolean arithmetic, shifts, logic, comparisons, conversions from floating
       point to integers (the Philox rounds are most of it); address arithmetic on pointers
       and conversions between integer types (truncations, extensions) are not counted;
  xu   calls of transcendental functions and square roots (sqrt, exp, log, sin, cos, tan,
       atan2, expm1, log1p, tanh, ...), each counted once;

and weighted by its block's count.  Loads, stores, copies and control flow are not counted.
The counts are per incident neutron of the sample, in total and per oracle function.

  python oracle/opcount.py [--workload powder_sqe] [--n N] [--out FILE]

Workloads: powder_sqe (the 100 meV powder S(Q,E) run), phonon_vanadium, bragg_aluminium,
dispersion_crystal (each through the bounded chain, orc_trace) and paper_powder_sqe (the
powder S(Q,E) run through the paper's recursive estimator, orc_trace_paper).
"""
from __future__ import annotations

import argparse
import ctypes as C
import glob
import json
import os
import re
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

FLAGS = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
         "-DORC_CONDITION=0"]

XU_FUNCS = {"sqrt", "exp", "log", "sin", "cos", "sincos", "tan", "atan2", "atan", "expm1",
            "log1p", "tanh", "pow", "cbrt", "acos", "asin", ".SQRT", "__builtin_sqrt",
            "hypot", "exp2", "log2"}
FP_FUNCS = {"fabs", "floor", "ceil", "fmin", "fmax", "trunc", "round", "copysign",
            ".COPYSIGN", ".FMIN", ".FMAX"}
FP_TYPES = ("double", "float", "long double")
OPS = re.compile(r"\s(\+|-|\*|/|%|&|\||\^|<<|>>|r<<|r>>|w\*|h\*|<=|>=|<|>|==|!=|u<=|u>=|u<|u>|"
                 r"uneq|unlt|unle|ungt|unge|ord|unord)\s")


# name -> (workload constructor of mcv_inputs, estimator, description)
WORKLOADS = {
    "powder_sqe": ("config2", "chain",
                   "config 2 powder S(Q,E) (hollow cylinder, 100 meV, up to 5 orders, "
                   "117,760-pixel tube system)"),
    "phonon_vanadium": ("vanadium_powder", "chain",
                        "vanadium-like hollow cylinder, incoherent phonon expansion from a DOS, "
                        "100 meV, up to 5 orders, 117,760-pixel tube system"),
    "bragg_aluminium": ("aluminium_powder", "chain",
                        "aluminium-like powder hollow cylinder, Debye-Scherrer reflections + "
                        "weak incoherent elastic, 100 meV, up to 5 orders"),
    "dispersion_crystal": ("dispersion_crystal", "chain",
                           "1 cm cube crystal, the paper's example dispersion surface, 7.5 meV, "
                           "up to 5 orders"),
    "paper_powder_sqe": ("config2", "paper",
                         "config 2 powder S(Q,E) through the paper's recursive estimator"),
}


def workload(name, n):
    sys.path.insert(0, ROOT)
    import mcv_inputs as mi
    make = getattr(mi, WORKLOADS[name][0])
    return make(n=n)


def _run_sample(lib_path, n, name="powder_sqe", first_id=0):
    """Runs the workload's first n neutrons through orc_trace (orc_trace_paper for the paper
    estimator) of lib_path, in this process: the profile counters are written when it
    exits."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle as O
    L = C.CDLL(lib_path)
    wl = workload(name, n)
    cfg = O.make_config(wl)
    hist = np.zeros(wl.detector.n_bins)
    tal = np.zeros(O.NTALLY)
    if WORKLOADS[name][1] == "paper":
        L.orc_trace_paper.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]
        L.orc_trace_paper.restype = C.c_int
        rc = L.orc_trace_paper(C.byref(cfg), first_id, n, hist.ctypes.data_as(C.c_void_p),
                               tal.ctypes.data_as(C.c_void_p))
    else:
        L.orc_trace.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p]
        L.orc_trace.restype = C.c_int
        rc = L.orc_trace(C.byref(cfg), first_id, n, None, None,
                         hist.ctypes.data_as(C.c_void_p), tal.ctypes.data_as(C.c_void_p))
    if rc:
        raise RuntimeError("the oracle's trace failed")
    return tal


def _types(fn_text):
    """name -> type of the declarations and parameters of one function's dump."""
    types = {}
    head = fn_text.split("\n{", 1)
    sig = head[0].splitlines()[-1] if head else ""
    m = re.search(r"\((.*)\)\s*$", sig)
    if m:
        for p in m.group(1).split(","):
            p = p.strip()
            mm = re.match(r"(.*?)([A-Za-z_][A-Za-z_0-9]*)$", p)
            if mm:
                types[mm.group(2)] = mm.group(1).strip()
    for line in fn_text.splitlines():
        mm = re.match(r"^  ([A-Za-z_][\w :<>*]*?)\s+\*?([A-Za-z_][\w.]*);$", line)
        if mm and "=" not in line:
            types[mm.group(2)] = mm.group(1).strip()
    return types


def _type_of(name, types):
    name = name.strip()
    name = re.sub(r"\(D\)$", "", name)
    if name in types:
        return types[name]
    base = re.sub(r"_\d+$", "", name)
    return types.get(base, "")


def _is_fp(t):
    return any(t.startswith(x) for x in FP_TYPES) and "*" not in t


def _is_ptr(t):
    return "*" in t


def _is_num(tok):
    return bool(re.match(r"^-?[\d.]+(e[+-]?\d+)?$", tok.strip()))


def _classify(stmt, types):
    """(fp, int, xu) operations of one GIMPLE statement."""
    s = stmt.strip().rstrip(";")
    if not s or s.startswith(("#", "goto", "return", "<", "//", "else", "switch")):
        return 0, 0, 0
    if s.startswith("if ("):
        cond = s[4:s.rfind(")")]
        m = OPS.search(" " + cond + " ")
        if not m:
            return 0, 0, 0
        lhs = (" " + cond + " ")[: m.start()].strip()
        t = _type_of(lhs, types)
        if not t and _is_num(lhs):
            rhs = (" " + cond + " ")[m.end():].strip()
            t = _type_of(rhs, types)
        return (1, 0, 0) if _is_fp(t) else (0, 1, 0)
    if "=" not in s or s.startswith("MEM") and " = " not in s:
        # a call without a result
        m = re.match(r"^([.\w]+) \(", s)
        if m and m.group(1) in XU_FUNCS:
            return 0, 0, 1
        return 0, 0, 0
    if " = " not in s:
        return 0, 0, 0
    lhs, rhs = s.split(" = ", 1)
    lhs = lhs.strip()
    t = _type_of(lhs, types)
    m = re.match(r"^([.\w]+) \((.*)\)$", rhs)
    if m and not rhs.startswith("("):
        f = m.group(1)
        if f in XU_FUNCS:
            return 0, 0, 1
        if f in FP_FUNCS:
            return 1, 0, 0
        return 0, 0, 0
    if re.match(r"^(ABS_EXPR|MIN_EXPR|MAX_EXPR|ABSU_EXPR)\s*<", rhs):
        return (1, 0, 0) if _is_fp(t) else (0, 1, 0)
    mc = re.match(r"^\([\w :<>*]+\) ([\w.()]+)$", rhs)
    if mc:                                                    # a conversion
        if _is_ptr(t):
            return 0, 0, 0
        if _is_fp(t):
            return 1, 0, 0
        # integer to integer (a truncation or an extension): no operation on a GPU or CPU
        src_t = _type_of(mc.group(1), types)
        return (0, 1, 0) if _is_fp(src_t) else (0, 0, 0)
    if rhs.startswith("-") and re.match(r"^-[A-Za-z_][\w.()]*$", rhs):   # negation
        return (1, 0, 0) if _is_fp(t) else (0, 1, 0)
    if rhs.startswith("~") or rhs.startswith("!"):
        return 0, 1, 0
    if " ? " in rhs:
        return (1, 0, 0) if _is_fp(t) else (0, 1, 0)
    mop = OPS.search(" " + rhs + " ")
    if mop:
        if _is_ptr(t):
            return 0, 0, 0
        op = mop.group(1)
        if op in ("<", ">", "<=", ">=", "==", "!=") or op.startswith(("u", "ord", "un")):
            a = (" " + rhs + " ")[: mop.start()].strip()
            ta = _type_of(a, types)
            return (1, 0, 0) if _is_fp(ta) else (0, 1, 0)
        return (1, 0, 0) if _is_fp(t) else (0, 1, 0)
    return 0, 0, 0


def parse_dump(text):
    """{function: [fp, int, xu]} weighted by block counts."""
    out = {}
    for chunk in text.split("\n;; Function ")[1:]:
        name = chunk.split(" ", 1)[0]
        types = _types(chunk)
        fp = it = xu = 0.0
        count = 0.0
        calls = None
        for line in chunk.splitlines():
            m = re.match(r"^;;\s+basic block \d+, loop depth \d+, count (\d+) \((\w+)", line)
            if m:
                # measured counts only (a function never run has none)
                count = float(m.group(1)) if m.group(2) in ("precise", "adjusted") else 0.0
                if calls is None:
                    calls = count  # the entry block: the calls of the function
                continue
            if re.match(r"^;;\s+basic block \d+", line):
                count = 0.0
                continue
            if line.startswith(";;") or not line.startswith("  ") or count == 0.0:
                continue
            a, b, c = _classify(line, types)
            fp += a * count
            it += b * count
            xu += c * count
        if fp or it or xu:
            out[name] = [fp, it, xu, calls or 0.0]
    return out


def count(n=100_000, name="powder_sqe"):
    src = os.path.join(HERE, "oracle.cpp")
    with tempfile.TemporaryDirectory() as d:
        obj = os.path.join(d, "oracle.o")
        lib1 = os.path.join(d, "liboracle_gen.so")
        # the profile is written next to the object (d/oracle.gcda) and read back by the
        # second compilation of the same object
        subprocess.run(FLAGS + ["-c", "-fprofile-generate", "-fprofile-update=single", "-o",
                                obj, src], check=True)
        subprocess.run(["g++", "-shared", "-fprofile-generate", "-o", lib1, obj], check=True)
        # run in a child process so that the profile is written at its exit
        code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); "
                "import opcount; t = opcount._run_sample(%r, %d, %r); "
                "import json; print(json.dumps(t.tolist()))" % (HERE, ROOT, lib1, n, name))
        r = subprocess.run([sys.executable, "-c", code], check=True, capture_output=True,
                           text=True)
        tallies = json.loads(r.stdout.strip().splitlines()[-1])
        if not os.path.exists(os.path.join(d, "oracle.gcda")):
            raise RuntimeError("no profile written")
        subprocess.run(FLAGS + ["-c", "-fprofile-use", "-fprofile-correction",
                                "-fdump-tree-optimized-details-blocks", "-dumpdir", d + "/",
                                "-o", obj, src], check=True, cwd=d)
        dumps = glob.glob(os.path.join(d, "*optimized"))
        if not dumps:
            raise RuntimeError("no GIMPLE dump")
        text = open(dumps[0]).read()
        if "(precise)" not in text:
            raise RuntimeError("the dump carries no measured block counts (profile not matched)")
    per_fn = parse_dump(text)
    tot = [sum(v[i] for v in per_fn.values()) for i in range(3)]
    return {"neutrons": n, "tallies": tallies,
            "per_neutron": {"fp": tot[0] / n, "int": tot[1] / n, "xu": tot[2] / n},
            "per_function_columns": ["fp per neutron", "int per neutron", "xu per neutron",
                                     "calls per neutron"],
            "per_function": {k: [v[0] / n, v[1] / n, v[2] / n, v[3] / n] for k, v in
                             sorted(per_fn.items(), key=lambda kv: -sum(kv[1][:3]))}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="powder_sqe", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    out = a.out or os.path.join(ROOT, "profiles", "opcount_%s.json" % a.workload)
    res = count(a.n, a.workload)
    res["command"] = "python oracle/opcount.py --workload %s --n %d" % (a.workload, a.n)
    res["workload"] = WORKLOADS[a.workload][2] + ", neutron ids 0..n-1"
    res["estimator"] = WORKLOADS[a.workload][1]
    with open(out, "w") as f:
        json.dump(res, f, indent=1)
    pn = res["per_neutron"]
    print("per neutron: fp %.1f  int %.1f  xu %.1f" % (pn["fp"], pn["int"], pn["xu"]))


if __name__ == "__main__":
    main()
