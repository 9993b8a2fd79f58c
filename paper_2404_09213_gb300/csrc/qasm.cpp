// OpenQASM 2.0 import and export for the subset of qelib1.inc gates this library simulates.
//
// The paper's simulator is built to exchange circuits with other platforms through this format
// (Sec. "API": export to OpenQASM). Import turns a program into the {type, targets, controls, param}
// records that qsim_plan takes: quantum registers are concatenated in declaration order into one
// qubit index space, and every rotation gets its own parameter slot holding its literal angle, so
// the circuit runs unchanged and its angles can then be trained. Export writes a gate list with
// given angles back as a program over one register q.
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace qsim {
void set_last_error(const std::string& s);
}

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Parser {
  const char* s;
  size_t i = 0, n = 0;
  int line = 1;
  std::string err;
  std::map<std::string, std::pair<int, int>> qregs;   // name -> (first qubit, size)
  std::map<std::string, int> cregs;
  int n_qubits = 0;
  std::vector<qsim_gate> gates;
  std::vector<double> params;

  int stmt_line = 1;   // errors name the line where the failing statement starts
  bool fail(const std::string& m) {
    if (err.empty()) err = "line " + std::to_string(stmt_line) + ": " + m;
    return false;
  }
  void skip() {   // whitespace and // comments
    for (;;) {
      while (i < n && std::isspace((unsigned char)s[i])) {
        if (s[i] == '\n') line++;
        i++;
      }
      if (i + 1 < n && s[i] == '/' && s[i + 1] == '/') {
        while (i < n && s[i] != '\n') i++;
        continue;
      }
      break;
    }
  }
  bool peek(char c) {
    skip();
    return i < n && s[i] == c;
  }
  bool eat(char c) {
    if (!peek(c)) return false;
    i++;
    return true;
  }
  bool expect(char c) { return eat(c) ? true : fail(std::string("expected '") + c + "'"); }
  std::string ident() {
    skip();
    size_t j = i;
    if (j < n && (std::isalpha((unsigned char)s[j]) || s[j] == '_')) {
      while (j < n && (std::isalnum((unsigned char)s[j]) || s[j] == '_')) j++;
    }
    std::string r(s + i, j - i);
    i = j;
    return r;
  }
  bool integer(long& v) {
    skip();
    size_t j = i;
    while (j < n && std::isdigit((unsigned char)s[j])) j++;
    if (j == i) return fail("expected an integer");
    v = std::strtol(std::string(s + i, j - i).c_str(), nullptr, 10);
    i = j;
    return true;
  }
  // expression := term (('+'|'-') term)*; term := unary (('*'|'/') unary)*;
  // unary := ('-'|'+') unary | number | 'pi' | '(' expression ')'
  bool expr(double& v) {
    if (!term(v)) return false;
    for (;;) {
      double r;
      if (eat('+')) {
        if (!term(r)) return false;
        v += r;
      } else if (eat('-')) {
        if (!term(r)) return false;
        v -= r;
      } else {
        return true;
      }
    }
  }
  bool term(double& v) {
    if (!unary(v)) return false;
    for (;;) {
      double r;
      if (eat('*')) {
        if (!unary(r)) return false;
        v *= r;
      } else if (eat('/')) {
        if (!unary(r)) return false;
        if (r == 0.0) return fail("division by zero in an angle");
        v /= r;
      } else {
        return true;
      }
    }
  }
  bool unary(double& v) {
    if (eat('-')) {
      if (!unary(v)) return false;
      v = -v;
      return true;
    }
    if (eat('+')) return unary(v);
    if (eat('(')) return expr(v) && expect(')');
    skip();
    if (i < n && (std::isdigit((unsigned char)s[i]) || s[i] == '.')) {
      char* end = nullptr;
      v = std::strtod(s + i, &end);
      if (end == s + i) return fail("bad number");
      i = (size_t)(end - s);
      return true;
    }
    const std::string id = ident();
    if (id == "pi") {
      v = kPi;
      return true;
    }
    return fail(id.empty() ? "expected an angle" : "unknown symbol '" + id + "' in an angle");
  }
  // one qubit argument: reg[i] or a whole register (size > 1 broadcasts)
  bool qarg(std::vector<int>& qs) {
    const std::string r = ident();
    auto it = qregs.find(r);
    if (it == qregs.end()) return fail(r.empty() ? "expected a qubit" : "unknown quantum register '" + r + "'");
    qs.clear();
    if (eat('[')) {
      long k;
      if (!integer(k) || !expect(']')) return false;
      if (k < 0 || k >= it->second.second) return fail("qubit index " + std::to_string(k) + " out of range");
      qs.push_back(it->second.first + (int)k);
    } else {
      for (int k = 0; k < it->second.second; k++) qs.push_back(it->second.first + k);
    }
    return true;
  }
  void push(int type, int t, int c, int param) {
    qsim_gate g;
    g.type = type;
    g.targets[0] = t;
    g.targets[1] = -1;
    g.controls[0] = c;
    g.controls[1] = -1;
    g.param = param;
    gates.push_back(g);
  }
  bool statement() {
    skip();
    stmt_line = line;
    const std::string kw = ident();
    if (kw.empty()) return fail("expected a statement");
    if (kw == "OPENQASM") {
      double v;
      if (!expr(v)) return false;
      if (v < 2.0 || v >= 3.0) return fail("only OpenQASM 2.x is supported");
      return expect(';');
    }
    if (kw == "include") {
      skip();
      if (i >= n || s[i] != '"') return fail("expected a file name");
      size_t j = s[i] == '"' ? i + 1 : i;
      while (j < n && s[j] != '"') j++;
      const std::string f(s + i + 1, j - i - 1);
      i = j + 1;
      if (f != "qelib1.inc") return fail("only qelib1.inc can be included");
      return expect(';');
    }
    if (kw == "qreg" || kw == "creg") {
      const std::string name = ident();
      long sz;
      if (name.empty()) return fail("expected a register name");
      if (!expect('[') || !integer(sz) || !expect(']') || !expect(';')) return false;
      if (sz < 1) return fail("register size must be >= 1");
      if (qregs.count(name) || cregs.count(name)) return fail("register '" + name + "' declared twice");
      if (kw == "qreg") {
        if (n_qubits + sz > 34) return fail("more than 34 qubits");
        qregs[name] = {n_qubits, (int)sz};
        n_qubits += (int)sz;
      } else {
        cregs[name] = (int)sz;
      }
      return true;
    }
    if (kw == "barrier") {   // no effect on the simulated state
      while (i < n && !peek(';')) i++;
      return expect(';');
    }
    if (kw == "measure") {   // results are <Z_i> of the final state; measurement records are ignored
      while (i < n && !peek(';')) i++;
      return expect(';');
    }
    struct G { int type, nq, angle; };
    static const std::map<std::string, G> known = {
        {"h", {QSIM_H, 1, 0}},   {"x", {QSIM_X, 1, 0}},     {"rx", {QSIM_RX, 1, 1}},
        {"ry", {QSIM_RY, 1, 1}}, {"rz", {QSIM_RZ, 1, 1}},   {"cx", {QSIM_CNOT, 2, 0}},
        {"CX", {QSIM_CNOT, 2, 0}}, {"cz", {QSIM_CZ, 2, 0}}, {"id", {-1, 1, 0}}};
    auto it = known.find(kw);
    if (it == known.end()) return fail("unsupported statement or gate '" + kw + "'");
    const G g = it->second;
    double angle = 0.0;
    if (g.angle) {
      if (!expect('(') || !expr(angle) || !expect(')')) return false;
    } else if (peek('(')) {
      return fail("gate '" + kw + "' takes no angle");
    }
    std::vector<int> a, b;
    if (!qarg(a)) return false;
    if (g.nq == 2 && (!expect(',') || !qarg(b))) return false;
    if (!expect(';')) return false;
    if (g.nq == 2) {   // registers broadcast pairwise; a single qubit pairs with every qubit of the other
      size_t m = std::max(a.size(), b.size());
      if ((a.size() != 1 && a.size() != m) || (b.size() != 1 && b.size() != m))
        return fail("registers of different sizes in '" + kw + "'");
      for (size_t k = 0; k < m; k++) {
        const int c = a[a.size() == 1 ? 0 : k], t = b[b.size() == 1 ? 0 : k];
        if (c == t) return fail("control and target are the same qubit");
        push(g.type, t, c, -1);
      }
      return true;
    }
    for (int q : a) {
      if (g.type < 0) continue;   // id
      if (g.angle) {
        push(g.type, q, -1, (int)params.size());
        params.push_back(angle);
      } else {
        push(g.type, q, -1, -1);
      }
    }
    return true;
  }
  bool program() {
    skip();
    while (i < n) {
      if (!statement()) return false;
      skip();
    }
    if (n_qubits == 0) return fail("no quantum register declared");
    return true;
  }
};

}  // namespace

extern "C" {

int qsim_parse_qasm(const char* text, qsim_gate* h_gates, int32_t cap_gates, int32_t* n_gates, double* h_params,
                    int32_t cap_params, int32_t* n_params, int32_t* n_qubits) {
  qsim::set_last_error("");
  if (!text || !n_gates || !n_params || !n_qubits) {
    qsim::set_last_error("qsim_parse_qasm: text and the three counts are required");
    return QSIM_ERR_ARG;
  }
  Parser p;
  p.s = text;
  p.n = std::strlen(text);
  if (!p.program()) {
    qsim::set_last_error("OpenQASM: " + p.err);
    return QSIM_ERR_ARG;
  }
  *n_gates = (int32_t)p.gates.size();
  *n_params = (int32_t)p.params.size();
  *n_qubits = p.n_qubits;
  if ((h_gates && cap_gates < *n_gates) || (h_params && cap_params < *n_params)) {
    qsim::set_last_error("qsim_parse_qasm: output arrays too small (need " + std::to_string(*n_gates) +
                         " gates, " + std::to_string(*n_params) + " parameters)");
    return QSIM_ERR_ARG;
  }
  if (h_gates) std::memcpy(h_gates, p.gates.data(), p.gates.size() * sizeof(qsim_gate));
  if (h_params) std::memcpy(h_params, p.params.data(), p.params.size() * sizeof(double));
  return QSIM_OK;
}

int qsim_export_qasm(const qsim_gate* h_gates, int32_t n_gates, int32_t n_qubits, const double* h_params,
                     const double* h_inputs, char* buf, size_t cap, size_t* needed) {
  qsim::set_last_error("");
  if ((!h_gates && n_gates > 0) || n_qubits < 1 || n_qubits > 34 || !needed) {
    qsim::set_last_error("qsim_export_qasm: bad arguments");
    return QSIM_ERR_ARG;
  }
  std::string out = "OPENQASM 2.0;\ninclude \"qelib1.inc\";\nqreg q[" + std::to_string(n_qubits) + "];\n";
  char line[160];
  for (int i = 0; i < n_gates; i++) {
    const qsim_gate& g = h_gates[i];
    const int t = g.targets[0], c = g.controls[0];
    if (t < 0 || t >= n_qubits) {
      qsim::set_last_error("qsim_export_qasm: gate " + std::to_string(i) + " has no valid target");
      return QSIM_ERR_QUBIT;
    }
    switch (g.type) {
      case QSIM_RX:
      case QSIM_RY:
      case QSIM_RZ: {
        double a;
        if (g.param >= 0) {
          if (!h_params) {
            qsim::set_last_error("qsim_export_qasm: parametric gate but h_params is NULL");
            return QSIM_ERR_ARG;
          }
          a = h_params[g.param];
        } else if (g.param <= -2) {
          if (!h_inputs) {
            qsim::set_last_error("qsim_export_qasm: input-encoded gate but h_inputs is NULL");
            return QSIM_ERR_ARG;
          }
          a = h_inputs[-2 - g.param];
        } else {
          qsim::set_last_error("qsim_export_qasm: rotation " + std::to_string(i) + " has no angle");
          return QSIM_ERR_PARAM;
        }
        const char* nm = g.type == QSIM_RX ? "rx" : g.type == QSIM_RY ? "ry" : "rz";
        std::snprintf(line, sizeof line, "%s(%.17g) q[%d];\n", nm, a, t);
        break;
      }
      case QSIM_H: std::snprintf(line, sizeof line, "h q[%d];\n", t); break;
      case QSIM_X: std::snprintf(line, sizeof line, "x q[%d];\n", t); break;
      case QSIM_CNOT:
      case QSIM_CZ:
        if (c < 0 || c >= n_qubits || c == t) {
          qsim::set_last_error("qsim_export_qasm: gate " + std::to_string(i) + " has no valid control");
          return QSIM_ERR_QUBIT;
        }
        std::snprintf(line, sizeof line, "%s q[%d],q[%d];\n", g.type == QSIM_CNOT ? "cx" : "cz", c, t);
        break;
      default:
        qsim::set_last_error("qsim_export_qasm: unknown gate type " + std::to_string(g.type));
        return QSIM_ERR_ARG;
    }
    out += line;
  }
  *needed = out.size() + 1;
  if (buf) {
    if (cap < *needed) {
      qsim::set_last_error("qsim_export_qasm: buffer too small");
      return QSIM_ERR_ARG;
    }
    std::memcpy(buf, out.c_str(), out.size() + 1);
  }
  return QSIM_OK;
}

}  // extern "C"
